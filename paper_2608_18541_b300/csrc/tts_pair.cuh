// tts_pair.cuh -- the FP32 spin update of two sites at once on the packed
// f32x2 pipe (add/sub/mul/fma .f32x2, one instruction for both lanes).
//
// A value f2 holds lane A in its low and lane B in its high 32 bits.  Every
// operation is lane-wise, and each lane's result depends on that lane's
// inputs only, so a site's trajectory does not depend on which site it is
// paired with.  Transcendentals (reciprocal square root, base-2 exponential
// and logarithm, reciprocal, sine and cosine) have no packed form and run per
// lane on the PTX approximate instructions.
//
// The sub-step map is the same exact frozen-field LLG flow (paper Eq. 1) as
// the scalar fast update:  with b = B/|B|, c = s.b, s_perp = s - c b,
// q = b x s, phi = gamma'|B| h, x = alpha phi, E = e^{-2x},
//   D = (1 + c) + (1 - c) E,  c' = ((1 + c) - (1 - c) E) / D,  rho = 2 e^{-x} / D,
//   s' = c' b + rho (cos(phi) s_perp + sin(phi) q),
// then renormalised; the on-site anisotropy field is taken at the predicted
// sub-step midpoint and the thermal field (Eq. 2) is sigma * g with g from a
// Box-Muller transform of one Philox4x32-10 block per site.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tts_fastmath.cuh"
#include "tts_philox.cuh"

namespace tts {

struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 f2_make(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(f2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f2 f2_swap(f2 a)
{
    float lo, hi;
    f2_split(a, lo, hi);
    return f2_make(hi, lo);
}
// lane A of a, lane B of b
__device__ __forceinline__ f2 f2_mix(f2 a, f2 b)
{
    float al, ah, bl, bh;
    f2_split(a, al, ah);
    f2_split(b, bl, bh);
    return f2_make(al, bh);
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
// a * b + c, one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// sine and cosine of an angle in (-pi, pi), the hardware approximations
__device__ __forceinline__ float sin_approx(float x)
{
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// lane-wise transcendental of an f2
template <float (*Fn)(float)>
__device__ __forceinline__ f2 f2_map(f2 a)
{
    float lo, hi;
    f2_split(a, lo, hi);
    return f2_make(Fn(lo), Fn(hi));
}

// Per-pass constants of the pair update, each a (species-0, species-1 minus
// species-0) couple so that a lane's value is c0 + w d with w = 0 / 1 the
// lane's species flag; all are lane-splatted.
struct PairConsts {
    f2 J0c, J0d;       // J(t_i, 0) / mu_i
    f2 dJc, dJd;       // (J(t_i, 1) - J(t_i, 0)) / mu_i
    f2 kc, kd;         // 2 K / mu_i
    f2 alc, ald;       // alpha
    f2 khgc, khgd;     // -kappa gamma' h / 2   (midpoint anisotropy)
    f2 ghc, ghd;       // gamma' h               (precession angle per tesla)
    f2 nalc, nald;     // -alpha log2(e)        (e^{-alpha phi} = 2^{nal phi})
    f2 nx, ny, nz;     // anisotropy axis
    f2 Bx, By, Bz;     // applied field (tesla)
    f2 one, neg1;
    f2 u_off;          // uniform = (1 + (k >> 9) 2^-23) + u_off, u_off = 2^-24 - 1 (exact)
    f2 m2ln2;          // -2 ln 2   (-2 ln u = -2 ln2 log2 u)
    f2 twopi, negpi;
    f2 s3, s5;         // sine Taylor coefficients -1/6, 1/120
    f2 c2, c4, c6;     // cosine Taylor coefficients -1/2, 1/24, -1/720
};

// Thermal-field directions of two sites: one Philox4x32-10 block per site,
// Box-Muller to (g1, g2, g3) = -(r01 cos a1, r01 sin a1, r23 cos a3) with
// r = sqrt(-2 ln u) and a = 2 pi u - pi (so that -cos a = cos 2 pi u).
__device__ __forceinline__ void pair_noise(const u32x4 &ctrA, const u32x4 &ctrB, const PhiloxRoundKeys &rk,
                                           const PairConsts &k, f2 &g1, f2 &g2, f2 &g3)
{
    const u32x4 rA = philox4x32_10(ctrA, rk);
    const u32x4 rB = philox4x32_10(ctrB, rk);
    // (1 + m 2^-23) - (1 - 2^-24) = (2m + 1) 2^-24 exactly, m = x >> 9
    auto one_m = [](uint32_t x) { return __uint_as_float(0x3F800000u | (x >> 9)); };
    const f2 u0 = f2_make(one_m(rA.x), one_m(rB.x)) + k.u_off;
    const f2 u1 = f2_make(one_m(rA.y), one_m(rB.y)) + k.u_off;
    const f2 u2 = f2_make(one_m(rA.z), one_m(rB.z)) + k.u_off;
    const f2 u3 = f2_make(one_m(rA.w), one_m(rB.w)) + k.u_off;
    // radius sqrt(l) = l rsqrt(l) with l = -2 ln u = -2 ln2 log2 u
    const f2 l0 = f2_map<lg2_approx>(u0) * k.m2ln2;
    const f2 l2 = f2_map<lg2_approx>(u2) * k.m2ln2;
    const f2 nr01 = (l0 * f2_map<rsqrt_approx>(l0)) * k.neg1;
    const f2 nr23 = (l2 * f2_map<rsqrt_approx>(l2)) * k.neg1;
    const f2 a1 = fma2(u1, k.twopi, k.negpi);
    const f2 a3 = fma2(u3, k.twopi, k.negpi);
    g1 = nr01 * f2_map<cos_approx>(a1);
    g2 = nr01 * f2_map<sin_approx>(a1);
    g3 = nr23 * f2_map<cos_approx>(a3);
}

// Two sites of one colour.  s = (x, y, z) of lanes A and B, ht / h1 the sums
// of all / species-1 neighbour spins, w the species flags; with noise, the
// thermal field sig * g (a lane with sig = 0 adds nothing).  Returns the new
// spins.
// h2: the pass runs for twice the step the constants were made for (the
// step-length terms gamma' h and kappa gamma' h / 2 doubled, which is exact).
template <bool AXZ>
__device__ __forceinline__ void pair_update(f2 &sx, f2 &sy, f2 &sz, f2 htx, f2 hty, f2 htz, f2 h1x, f2 h1y, f2 h1z,
                                            f2 w, bool noise, f2 sig, f2 g1, f2 g2, f2 g3, const PairConsts &k,
                                            bool h2)
{
    const f2 J0 = fma2(w, k.J0d, k.J0c);
    const f2 dJ = fma2(w, k.dJd, k.dJc);
    const f2 kap = fma2(w, k.kd, k.kc);
    const f2 al = fma2(w, k.ald, k.alc);
    f2 khg = fma2(w, k.khgd, k.khgc);
    f2 gh = fma2(w, k.ghd, k.ghc);
    if (h2) {
        khg = khg + khg;
        gh = gh + gh;
    }
    const f2 nal = fma2(w, k.nald, k.nalc);
    const f2 cn0 = AXZ ? sz : fma2(sz, k.nz, fma2(sy, k.ny, sx * k.nx));
    const f2 ka = kap * cn0;
    f2 Bx, By, Bz;
    if (AXZ) {
        Bx = fma2(J0, htx, fma2(dJ, h1x, k.Bx));
        By = fma2(J0, hty, fma2(dJ, h1y, k.By));
        Bz = fma2(J0, htz, fma2(dJ, h1z, ka + k.Bz));
    } else {
        Bx = fma2(J0, htx, fma2(dJ, h1x, fma2(ka, k.nx, k.Bx)));
        By = fma2(J0, hty, fma2(dJ, h1y, fma2(ka, k.ny, k.By)));
        Bz = fma2(J0, htz, fma2(dJ, h1z, fma2(ka, k.nz, k.Bz)));
    }
    if (noise) {
        Bx = fma2(sig, g1, Bx);
        By = fma2(sig, g2, By);
        Bz = fma2(sig, g3, Bz);
    }
    // on-site anisotropy at the predicted sub-step midpoint
    if (AXZ) {
        const f2 n_sxB = sx * By - sy * Bx;
        const f2 sB = fma2(sz, Bz, fma2(sy, By, sx * Bx));
        Bz = fma2(khg, fma2(al, cn0 * sB - Bz, n_sxB), Bz);
    } else {
        const f2 cx = sy * Bz - sz * By, cy = sz * Bx - sx * Bz, cz = sx * By - sy * Bx;
        const f2 n_sxB = fma2(k.nz, cz, fma2(k.ny, cy, k.nx * cx));
        const f2 sB = fma2(sz, Bz, fma2(sy, By, sx * Bx));
        const f2 nB = fma2(k.nz, Bz, fma2(k.ny, By, k.nx * Bx));
        const f2 corr = khg * fma2(al, cn0 * sB - nB, n_sxB);
        Bx = fma2(corr, k.nx, Bx);
        By = fma2(corr, k.ny, By);
        Bz = fma2(corr, k.nz, Bz);
    }
    const f2 B2 = fma2(Bz, Bz, fma2(By, By, Bx * Bx));
    const f2 rb = f2_map<rsqrt_approx>(B2);
    const f2 bx = Bx * rb, by = By * rb, bz = Bz * rb;
    const f2 Bm = B2 * rb;
    const f2 c = fma2(sz, bz, fma2(sy, by, sx * bx));
    const f2 nc = c * k.neg1;
    const f2 px = fma2(nc, bx, sx), py = fma2(nc, by, sy), pz = fma2(nc, bz, sz);
    const f2 qx = by * sz - bz * sy, qy = bz * sx - bx * sz, qz = bx * sy - by * sx;
    const f2 phi = Bm * gh;
    const f2 em = f2_map<ex2_approx>(nal * phi);
    const f2 E = em * em;
    const f2 opc = k.one + c, omc = k.one - c;
    const f2 omcE = omc * E;
    const f2 iD = f2_map<rcp_approx>(opc + omcE);
    const f2 cp = (opc - omcE) * iD;
    const f2 rho = (em + em) * iD;
    // sin / cos of phi: Taylor through phi^5 / phi^6 below 1/4 rad (the
    // truncation, below phi^7 / 7! = 1.2e-8 there, is under one FP32 ulp of
    // sin phi).  Thermal fields of a few thousand kelvin give sub-step angles
    // of 0.02 to 0.2 rad.
    const f2 p2 = phi * phi;
    f2 sn = phi * fma2(p2, fma2(p2, k.s5, k.s3), k.one);
    f2 cs = fma2(p2, fma2(p2, fma2(p2, k.c6, k.c4), k.c2), k.one);
    float phA, phB, b2A, b2B;
    f2_split(phi, phA, phB);
    f2_split(B2, b2A, b2B);
    // one rarely taken branch for a large angle or a vanishing field in either lane
    const bool slow = !(phA < 0.25f && phB < 0.25f && b2A > 1e-30f && b2B > 1e-30f);
    if (slow) {
        float snA, snB, csA, csB;
        f2_split(sn, snA, snB);
        f2_split(cs, csA, csB);
        if (!(phA < 0.25f)) sincosf(phA, &snA, &csA);
        if (!(phB < 0.25f)) sincosf(phB, &snB, &csB);
        sn = f2_make(snA, snB);
        cs = f2_make(csA, csB);
    }
    const f2 ra = rho * cs, rbq = rho * sn;
    const f2 ox = fma2(rbq, qx, fma2(ra, px, cp * bx));
    const f2 oy = fma2(rbq, qy, fma2(ra, py, cp * by));
    const f2 oz = fma2(rbq, qz, fma2(ra, pz, cp * bz));
    const f2 on = f2_map<rsqrt_approx>(fma2(oz, oz, fma2(oy, oy, ox * ox)));
    f2 nx_ = ox * on, ny_ = oy * on, nz_ = oz * on;
    // a lane with no field (|B|^2 <= 1e-30 T^2: the precession angle of a
    // sub-step is below 1e-20 rad) keeps its spin
    if (slow) {
        float oA, oB, nA, nB;
        f2 *outs[3] = {&nx_, &ny_, &nz_};
        const f2 ins[3] = {sx, sy, sz};
        for (int j = 0; j < 3; ++j) {
            f2_split(ins[j], oA, oB);
            f2_split(*outs[j], nA, nB);
            *outs[j] = f2_make(b2A > 1e-30f ? nA : oA, b2B > 1e-30f ? nB : oB);
        }
    }
    sx = nx_;
    sy = ny_;
    sz = nz_;
}

}  // namespace tts
