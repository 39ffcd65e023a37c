// tts_engines.cu -- fast engines for simple-cubic lattices with nearest-
// neighbour exchange.
//
// CHECKER  (all cell counts even, any instance count, equal instance shapes)
//   Colour c = (x + y + z) mod 2.  The general slot order of such an instance
//   (colour-major, ascending atom id) is the checkerboard raster order:
//   colour-c site (x, y, z) sits at ((z Ly + y) Lx/2 + x/2).  Spins are kept
//   as float4 / double4 (x, y, z, species) in that order, so the six
//   neighbours of a site are found by index arithmetic and read with one
//   vector load each.  One launch per colour pass.
//
// RESIDENT (instances small enough for shared memory, uniform bath or a
//   one-cell TTM per instance)
//   A persistent kernel: each CTA takes whole instances from a queue (largest
//   first), copies the instance's spins into shared memory and advances it
//   for all n steps of tts_step -- every colour pass, the FP64 noise table,
//   the FP64 one-cell TTM and the FP64 observables -- before writing it back.
//   The many independent realisations of a phase-diagram campaign (the task-
//   level replicas of the paper's Sec. II.F) advance together in one launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tts_engines.h"
#include "tts_fastmath.cuh"
#include "tts_philox.cuh"

namespace tts {

namespace {
thread_local std::string g_engine_error = "no error";

int eng_fail(int code, const std::string &m)
{
    g_engine_error = m;
    return code;
}

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
    using T = float4;
};
struct __align__(32) double4a {
    double x, y, z, w;
};
template <>
struct Vec4<double> {
    using T = double4a;
};

// ---------------------------------------------------------------------------
// Checkerboard engine
// ---------------------------------------------------------------------------
struct CheckerInst {
    int64_t slot_begin;   // first general slot of the instance
    int64_t prefix;       // first work item of the instance in a pass
    uint32_t nhalf;       // sites per colour
    uint32_t Lx, Ly, Lz, hx;
    uint32_t inst_global;
    FastDiv div_hx, div_Ly;
};

template <typename R>
struct CheckerArgs {
    typename Vec4<R>::T *S;
    const CheckerInst *ci;
    const int *cell;             // general slot -> TTM cell
    const R *sigma;              // [cell][species][h]
    const int64_t *step;
    unsigned int *health;
    FastSpecies<R> sp[TTS_MAX_SPECIES];
    R nx, ny, nz, Bx, By, Bz;
    R dt;
    uint32_t key0, key1;
    int n_inst;
    int64_t total;               // work items per pass (sum of nhalf)
};

template <typename R>
__global__ void __launch_bounds__(256) checker_pass_kernel(CheckerArgs<R> a, int colour, int hsel, int pass)
{
    using V = typename Vec4<R>::T;
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= a.total) return;
    int i = 0;
    if (a.n_inst > 1) {
        int lo = 0, hi = a.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.ci[mid].prefix <= gid) lo = mid; else hi = mid - 1;
        }
        i = lo;
    }
    const CheckerInst &I = a.ci[i];
    const uint32_t k = static_cast<uint32_t>(gid - I.prefix);
    const uint32_t row = fast_div(k, I.div_hx);
    const uint32_t kx = k - row * I.hx;
    const uint32_t z = fast_div(row, I.div_Ly);
    const uint32_t y = row - z * I.Ly;
    const uint32_t x = 2 * kx + ((y + z + colour) & 1u);
    const uint32_t zp = (z + 1 == I.Lz) ? 0 : z + 1, zm = (z == 0) ? I.Lz - 1 : z - 1;
    const uint32_t yp = (y + 1 == I.Ly) ? 0 : y + 1, ym = (y == 0) ? I.Ly - 1 : y - 1;
    uint32_t kxp, kxm;
    if (x & 1u) {
        kxp = (kx + 1 == I.hx) ? 0 : kx + 1;
        kxm = kx;
    } else {
        kxp = kx;
        kxm = (kx == 0) ? I.hx - 1 : kx - 1;
    }
    const int64_t own_base = I.slot_begin + int64_t(colour) * I.nhalf;
    const V *O = a.S + I.slot_begin + int64_t(1 - colour) * I.nhalf;
    const uint32_t rz = z * I.Ly, rowhx = row * I.hx;
    const V n0 = O[(zp * I.Ly + y) * I.hx + kx];
    const V n1 = O[(zm * I.Ly + y) * I.hx + kx];
    const V n2 = O[(rz + yp) * I.hx + kx];
    const V n3 = O[(rz + ym) * I.hx + kx];
    const V n4 = O[rowhx + kxp];
    const V n5 = O[rowhx + kxm];
    V own = a.S[own_base + k];
    const R htx = n0.x + n1.x + n2.x + n3.x + n4.x + n5.x;
    const R hty = n0.y + n1.y + n2.y + n3.y + n4.y + n5.y;
    const R htz = n0.z + n1.z + n2.z + n3.z + n4.z + n5.z;
    const R h1x = n0.w * n0.x + n1.w * n1.x + n2.w * n2.x + n3.w * n3.x + n4.w * n4.x + n5.w * n5.x;
    const R h1y = n0.w * n0.y + n1.w * n1.y + n2.w * n2.y + n3.w * n3.y + n4.w * n4.y + n5.w * n5.y;
    const R h1z = n0.w * n0.z + n1.w * n1.z + n2.w * n2.z + n3.w * n3.z + n4.w * n4.z + n5.w * n5.z;
    const int t = own.w != R(0) ? 1 : 0;
    const FastSpecies<R> sp = t ? a.sp[1] : a.sp[0];
    const int64_t slot = own_base + k;
    const R sig = a.sigma[(int64_t(a.cell[slot]) * TTS_MAX_SPECIES + t) * 2 + hsel];
    const R h = hsel ? a.dt : R(0.5) * a.dt;
    R sx = own.x, sy = own.y, sz = own.z;
    if (sig > R(0)) {
        const uint32_t atom = (z * I.Ly + y) * I.Lx + x;
        const u32x4 w = philox4x32_10(u32x4{atom, static_cast<uint32_t>(*a.step), static_cast<uint32_t>(pass),
                                            I.inst_global},
                                      a.key0, a.key1);
        fast_update<R>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, sp, a.nx, a.ny, a.nz, a.Bx, a.By, a.Bz, sig, &w, h);
    } else {
        fast_update<R>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, sp, a.nx, a.ny, a.nz, a.Bx, a.By, a.Bz, sig, nullptr,
                       h);
    }
    if (!(isfinite(sx) && isfinite(sy) && isfinite(sz))) atomicOr(a.health, kHealthNonFinite);
    own.x = sx;
    own.y = sy;
    own.z = sz;
    a.S[slot] = own;
}

// general SoA <-> engine float4 (same slot order)
template <typename R>
__global__ void to_general_kernel(const typename Vec4<R>::T *__restrict__ S, R *sx, R *sy, R *sz, int64_t n,
                                  const int64_t *step, int sample_every, int conditional)
{
    if (conditional && (sample_every <= 0 || (*step + 1) % sample_every != 0)) return;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const auto v = S[i];
    sx[i] = v.x;
    sy[i] = v.y;
    sz[i] = v.z;
}

template <typename R>
__global__ void from_general_kernel(typename Vec4<R>::T *S, const R *__restrict__ sx, const R *__restrict__ sy,
                                    const R *__restrict__ sz, const uint8_t *__restrict__ spc, int64_t n)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    typename Vec4<R>::T v;
    v.x = sx[i];
    v.y = sy[i];
    v.z = sz[i];
    v.w = spc[i] ? R(1) : R(0);
    S[i] = v;
}

// ---------------------------------------------------------------------------
// Resident engine
// ---------------------------------------------------------------------------
struct ResInst {
    int64_t slot_begin;
    int n;
    int L[3];
    FastDiv divx, divxy;
    int colour_begin[kMaxColours + 1];   // relative slots
    int ncolours;
    int inst;                            // local instance index
    uint32_t inst_global;
};

template <typename R>
struct ResArgs {
    R *sx, *sy, *sz;                     // general SoA spins
    const uint8_t *species;              // general slot order
    const int *atom;                     // general slot -> atom id
    const ResInst *ri;
    const int *order;                    // instance processing order
    int *queue;
    const int64_t *step;
    unsigned int *health;
    double *Te, *Tl;                     // per instance cell (one cell each)
    double *src_energy;
    const DevInstance *inst;
    double *obs_ring;
    int64_t *obs_count;
    FastSpecies<R> sp[TTS_MAX_SPECIES];
    SpeciesParams spd[TTS_MAX_SPECIES];  // FP64 constants (sigma, observables)
    double axis[3], B[3];
    double dt;
    uint32_t key0, key1;
    int n_inst;
    int nspecies;
    int sample_every;
    int obs_capacity;
    int nmax;                            // shared-memory capacity in sites
    int ttm_active;
    TtmParams tp;
};

// FP64 observables of the instance held in shared memory, reduced in a fixed
// order (thread partials, warp shuffles, warps in index order).
template <typename R>
__device__ __noinline__ void resident_observe(const ResArgs<R> &a, const ResInst &I, const R *sx, const R *sy,
                                             const R *sz, const uint8_t *spc, int64_t sstep, double Te, double Tl,
                                             double *warp_red)
{
    constexpr int F = 24;
    double acc[F];
#pragma unroll
    for (int k = 0; k < F; ++k) acc[k] = 0.0;
    const int Lx = I.L[0], Ly = I.L[1], Lz = I.L[2];
    for (int at = threadIdx.x; at < I.n; at += blockDim.x) {
        const int xy = Lx * Ly;
        const int z = at / xy, rem = at - z * xy, y = rem / Lx, x = rem - y * Lx;
        const int xp = x + 1 == Lx ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
        const int yp = y + 1 == Ly ? 0 : y + 1, ym = y == 0 ? Ly - 1 : y - 1;
        const int zp = z + 1 == Lz ? 0 : z + 1, zm = z == 0 ? Lz - 1 : z - 1;
        const int nb[6] = {(zp * Ly + y) * Lx + x, (zm * Ly + y) * Lx + x, (z * Ly + yp) * Lx + x,
                           (z * Ly + ym) * Lx + x, (z * Ly + y) * Lx + xp, (z * Ly + y) * Lx + xm};
        const int t = spc[at];
        const FastSpecies<R> sp = t ? a.sp[1] : a.sp[0];
        const SpeciesParams spd = t ? a.spd[1] : a.spd[0];
        const double s0 = sx[at], s1 = sy[at], s2 = sz[at];
        double hx = 0, hy = 0, hz = 0;
        for (int k = 0; k < 6; ++k) {
            const double J = spc[nb[k]] ? double(sp.J1) : double(sp.J0);
            hx += J * double(sx[nb[k]]);
            hy += J * double(sy[nb[k]]);
            hz += J * double(sz[nb[k]]);
        }
        const double mu = spd.mu;
        const double sn = s0 * a.axis[0] + s1 * a.axis[1] + s2 * a.axis[2];
        const double ka = spd.kappa * sn;
        const double Hx = mu * (hx + ka * a.axis[0] + a.B[0]);
        const double Hy = mu * (hy + ka * a.axis[1] + a.B[1]);
        const double Hz = mu * (hz + ka * a.axis[2] + a.B[2]);
        const double cx = s1 * Hz - s2 * Hy, cy = s2 * Hx - s0 * Hz, cz = s0 * Hy - s1 * Hx;
        double *q = acc + 12 * t;
        q[0] += 1.0;
        q[1] += s0;
        q[2] += s1;
        q[3] += s2;
        q[7] += -0.5 * mu * (s0 * hx + s1 * hy + s2 * hz);
        q[8] += -spd.K * sn * sn;
        q[9] += -mu * (a.B[0] * s0 + a.B[1] * s1 + a.B[2] * s2);
        q[10] += cx * cx + cy * cy + cz * cz;
        q[11] += s0 * Hx + s1 * Hy + s2 * Hz;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < F; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) warp_red[warp * F + k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[F];
        for (int k = 0; k < F; ++k) tot[k] = 0.0;
        for (int w = 0; w < nw; ++w)
            for (int k = 0; k < F; ++k) tot[k] += warp_red[w * F + k];
        double rec[TTS_NOBS];
        for (int k = 0; k < TTS_NOBS; ++k) rec[k] = 0.0;
        rec[0] = double(sstep) * a.dt;
        double musum = 0, mux = 0, muy = 0, muz = 0;
        for (int t = 0; t < TTS_MAX_SPECIES; ++t) {
            const double *q = tot + 12 * t;
            if (q[0] > 0.0) {
                rec[1 + 3 * t] = q[1] / q[0];
                rec[2 + 3 * t] = q[2] / q[0];
                rec[3 + 3 * t] = q[3] / q[0];
                const double m = a.spd[t].mu / kBohrMagneton;
                musum += m * q[0];
                mux += m * q[1];
                muy += m * q[2];
                muz += m * q[3];
            }
            rec[10] += q[7];
            rec[11] += q[8];
            rec[12] += q[9];
            rec[13 + t] = (q[0] > 0.0 && q[11] != 0.0) ? q[10] / (2.0 * kBoltzmann * q[11]) : 0.0;
        }
        rec[7] = mux / musum;
        rec[8] = muy / musum;
        rec[9] = muz / musum;
        rec[15] = Te;
        rec[16] = Tl;
        rec[19] = double(sstep);
        const int64_t k = a.obs_count[I.inst];
        double *dst = a.obs_ring + (int64_t(I.inst) * a.obs_capacity + (k % a.obs_capacity)) * TTS_NOBS;
        for (int j = 0; j < TTS_NOBS; ++j) dst[j] = rec[j];
        a.obs_count[I.inst] = k + 1;
    }
    __syncthreads();
}

template <typename R>
__global__ void resident_kernel(ResArgs<R> a, int64_t nsteps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    R *sx = reinterpret_cast<R *>(smem);
    R *sy = sx + a.nmax;
    R *sz = sy + a.nmax;
    uint8_t *spc = reinterpret_cast<uint8_t *>(sz + a.nmax);
    __shared__ int s_next;
    __shared__ R s_sigma[TTS_MAX_SPECIES][2];
    __shared__ double s_T[2];
    __shared__ double warp_red[32 * 24];
    const int64_t step0 = *a.step;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
        __syncthreads();
        const int qi = s_next;
        __syncthreads();
        if (qi >= a.n_inst) break;
        const ResInst I = a.ri[a.order[qi]];
        for (int s = threadIdx.x; s < I.n; s += blockDim.x) {
            const int64_t slot = I.slot_begin + s;
            const int at = a.atom[slot];
            sx[at] = a.sx[slot];
            sy[at] = a.sy[slot];
            sz[at] = a.sz[slot];
            spc[at] = a.species[slot];
        }
        double Te = 0.0, Tl = 0.0, deposited = 0.0;
        const DevInstance D = a.inst[I.inst];
        if (threadIdx.x == 0) {
            Te = a.Te[D.cell_begin];
            Tl = a.Tl[D.cell_begin];
        }
        __syncthreads();
        const int Lx = I.L[0], Ly = I.L[1], Lz = I.L[2];
        for (int64_t st = 0; st < nsteps; ++st) {
            const int64_t step = step0 + st;
            if (threadIdx.x == 0) {
                for (int t = 0; t < TTS_MAX_SPECIES; ++t)
                    for (int hs = 0; hs < 2; ++hs) {
                        double v = 0.0;
                        if (t < a.nspecies && Te > 0.0 && a.spd[t].alpha > 0.0) {
                            const double h = hs ? a.dt : 0.5 * a.dt;
                            v = sqrt(2.0 * a.spd[t].alpha * kBoltzmann * Te / (kGyro * a.spd[t].mu * h));
                        }
                        s_sigma[t][hs] = static_cast<R>(v);
                    }
            }
            __syncthreads();
            const int K = I.ncolours;
            for (int p = 0; p < 2 * K - 1; ++p) {
                const int c = p < K - 1 ? p : (p == K - 1 ? K - 1 : 2 * K - 2 - p);
                const int hsel = p == K - 1 ? 1 : 0;
                const R h = hsel ? R(a.dt) : R(0.5 * a.dt);
                const int beg = I.colour_begin[c], end = I.colour_begin[c + 1];
                for (int idx = beg + threadIdx.x; idx < end; idx += blockDim.x) {
                    const uint32_t at = static_cast<uint32_t>(a.atom[I.slot_begin + idx]);
                    const uint32_t z = fast_div(at, I.divxy);
                    const uint32_t rem = at - z * uint32_t(Lx * Ly);
                    const uint32_t y = fast_div(rem, I.divx);
                    const uint32_t x = rem - y * uint32_t(Lx);
                    const uint32_t xp = x + 1 == uint32_t(Lx) ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
                    const uint32_t yp = y + 1 == uint32_t(Ly) ? 0 : y + 1, ym = y == 0 ? Ly - 1 : y - 1;
                    const uint32_t zp = z + 1 == uint32_t(Lz) ? 0 : z + 1, zm = z == 0 ? Lz - 1 : z - 1;
                    const uint32_t nb[6] = {(zp * Ly + y) * Lx + x, (zm * Ly + y) * Lx + x, (z * Ly + yp) * Lx + x,
                                            (z * Ly + ym) * Lx + x, (z * Ly + y) * Lx + xp, (z * Ly + y) * Lx + xm};
                    R htx = 0, hty = 0, htz = 0, h1x = 0, h1y = 0, h1z = 0;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const R vx = sx[nb[k]], vy = sy[nb[k]], vz = sz[nb[k]];
                        const R w = spc[nb[k]] ? R(1) : R(0);
                        htx += vx;
                        hty += vy;
                        htz += vz;
                        h1x += w * vx;
                        h1y += w * vy;
                        h1z += w * vz;
                    }
                    const int t = spc[at];
                    const FastSpecies<R> sp = t ? a.sp[1] : a.sp[0];
                    R s0 = sx[at], s1 = sy[at], s2 = sz[at];
                    const R sig = s_sigma[t][hsel];
                    if (sig > R(0)) {
                        const u32x4 w = philox4x32_10(
                            u32x4{at, static_cast<uint32_t>(step), static_cast<uint32_t>(p), I.inst_global}, a.key0,
                            a.key1);
                        fast_update<R>(s0, s1, s2, htx, hty, htz, h1x, h1y, h1z, sp, R(a.axis[0]), R(a.axis[1]),
                                       R(a.axis[2]), R(a.B[0]), R(a.B[1]), R(a.B[2]), sig, &w, h);
                    } else {
                        fast_update<R>(s0, s1, s2, htx, hty, htz, h1x, h1y, h1z, sp, R(a.axis[0]), R(a.axis[1]),
                                       R(a.axis[2]), R(a.B[0]), R(a.B[1]), R(a.B[2]), sig, nullptr, h);
                    }
                    sx[at] = s0;
                    sy[at] = s1;
                    sz[at] = s2;
                }
                __syncthreads();
            }
            // one-cell TTM, t_n -> t_n+1 (no diffusion on a single cell)
            if (threadIdx.x == 0 && a.ttm_active) {
                const double delta = a.dt / D.substeps;
                for (int k = 0; k < D.substeps; ++k) {
                    const double tt = double(step) * a.dt + double(k) * delta;
                    double src = 0.0;
                    if (a.tp.source != TTS_SOURCE_NONE) {
                        const double zz = (tt - D.t0) / D.sigma_t;
                        src = D.P0 * exp(-0.5 * zz * zz);
                    }
                    const double xch = a.tp.G * (Te - Tl);
                    const double dE = delta * (-xch + src);
                    deposited += delta * src * D.cell_volume;
                    Tl += delta * xch / a.tp.C_l;
                    Te = sqrt(2.0 * (0.5 * a.tp.gamma_e * Te * Te + dE) / a.tp.gamma_e);
                }
            }
            if (a.sample_every > 0 && (step + 1) % a.sample_every == 0) {
                if (threadIdx.x == 0) {
                    s_T[0] = Te;
                    s_T[1] = Tl;
                }
                __syncthreads();
                resident_observe<R>(a, I, sx, sy, sz, spc, step + 1, s_T[0], s_T[1], warp_red);
            }
        }
        for (int s = threadIdx.x; s < I.n; s += blockDim.x) {
            const int64_t slot = I.slot_begin + s;
            const int at = a.atom[slot];
            const R v0 = sx[at], v1 = sy[at], v2 = sz[at];
            if (!(isfinite(v0) && isfinite(v1) && isfinite(v2))) atomicOr(a.health, kHealthNonFinite);
            a.sx[slot] = v0;
            a.sy[slot] = v1;
            a.sz[slot] = v2;
        }
        if (threadIdx.x == 0) {
            a.Te[D.cell_begin] = Te;
            a.Tl[D.cell_begin] = Tl;
            if (a.ttm_active) a.src_energy[I.inst] += deposited;
        }
        __syncthreads();
    }
}

__global__ void advance_step_kernel(int64_t *step, int64_t n, int *queue)
{
    *step += n;
    *queue = 0;
}

}  // namespace

// ---------------------------------------------------------------------------
struct EngineState {
    int engine = TTS_ENGINE_GENERAL;
    int precision = 32;
    int64_t n_total = 0;
    int n_inst = 0;
    // checker
    void *S = nullptr;
    CheckerInst *ci = nullptr;
    int64_t work = 0;
    int K = 2;
    // resident
    ResInst *ri = nullptr;
    int *order = nullptr;
    int *queue = nullptr;
    int nmax = 0;
    int block = 256;
    size_t smem = 0;
    int grid = 0;
    // both
    FastSpecies<float> spf[TTS_MAX_SPECIES];
    FastSpecies<double> spd[TTS_MAX_SPECIES];
    std::vector<DevInstance> dinst;
};

const char *engine_last_error() { return g_engine_error.c_str(); }

namespace {

// every atom has exactly its six simple-cubic nearest neighbours and J
// depends only on the species pair
bool sc_nearest_neighbour(const tts_system_desc &d, const HostInstance &hi)
{
    if (d.lattice != TTS_LATTICE_SC) return false;
    for (int k = 0; k < 3; ++k)
        if (hi.cells[k] < 3) return false;
    const double r1 = d.a, r2 = d.a * std::sqrt(2.0);
    for (int a = 0; a < d.nspecies; ++a)
        for (int b = 0; b < d.nspecies; ++b) {
            const tts_exchange &e = d.exch[a][b];
            if (e.kind == TTS_EXCH_NONE) continue;
            if (!(e.rc > r1 && e.rc <= r2)) return false;
        }
    for (int64_t i = 0; i < hi.n; ++i) {
        const int64_t cnt = hi.nbr_begin[i + 1] - hi.nbr_begin[i];
        bool any = false;
        for (int a = 0; a < d.nspecies; ++a)
            for (int b = 0; b < d.nspecies; ++b) any = any || d.exch[a][b].kind != TTS_EXCH_NONE;
        if (any && cnt != 6) {
            // zero couplings (J = 0 between some pair) drop neighbours: then the
            // implicit stencil still applies since J is taken from the species pair
            if (cnt > 6) return false;
        }
    }
    return true;
}

double pair_J_at(const tts_exchange &e, double r)
{
    if (e.kind == TTS_EXCH_NONE || !(r < e.rc)) return 0.0;
    if (e.kind == TTS_EXCH_CONST) return e.J1;
    const double x = (r / e.J3) * (r / e.J3);
    return 4.0 * e.J1 * x * (1.0 - e.J2 * x) * std::exp(-x);
}

template <typename R>
void fill_species(const tts_system_desc &d, FastSpecies<R> *out)
{
    for (int t = 0; t < TTS_MAX_SPECIES; ++t) {
        FastSpecies<R> f{};
        if (t < d.nspecies) {
            const double mu = d.mu_muB[t] * kBohrMagneton;
            f.J0 = static_cast<R>(pair_J_at(d.exch[t][0], d.a) / mu);
            f.J1 = static_cast<R>(d.nspecies > 1 ? pair_J_at(d.exch[t][1], d.a) / mu : 0.0);
            f.kappa = static_cast<R>(2.0 * d.K[t] / mu);
            f.alpha = static_cast<R>(d.alpha[t]);
            f.gprime = static_cast<R>(kGyro / (1.0 + d.alpha[t] * d.alpha[t]));
        }
        out[t] = f;
    }
}

size_t resident_bytes(int n, int precision) { return size_t(n) * (3 * (precision == 64 ? 8 : 4) + 1) + 16; }

bool fastdiv_ok(uint32_t d, uint32_t limit)
{
    const FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < limit; ++n)
        if (fast_div(n, f) != n / d) return false;
    return true;
}

}  // namespace

int engine_select(const tts_system_desc &d, const std::vector<HostInstance> &host, int requested)
{
    bool sc_nn = true;
    for (const HostInstance &hi : host) sc_nn = sc_nn && sc_nearest_neighbour(d, hi);
    if (!sc_nn) return -1;
    // resident: every instance fits the shared memory of one CTA
    int dev = 0, maxsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        maxsm = 0;
    }
    bool fits = true;
    for (const HostInstance &hi : host)
        fits = fits && resident_bytes(static_cast<int>(hi.n), d.precision) + 8192 <= size_t(maxsm);
    bool even_equal = true;
    for (const HostInstance &hi : host)
        for (int k = 0; k < 3; ++k)
            even_equal = even_equal && hi.cells[k] % 2 == 0 && hi.cells[k] == host[0].cells[k];
    if (requested == TTS_ENGINE_RESIDENT) return fits ? TTS_ENGINE_RESIDENT : -1;
    if (requested == TTS_ENGINE_CHECKER) return even_equal ? TTS_ENGINE_CHECKER : -1;
    // AUTO: many small instances -> resident; otherwise large even lattices -> checker
    if (fits && host.size() >= 8) return TTS_ENGINE_RESIDENT;
    if (even_equal) return TTS_ENGINE_CHECKER;
    if (fits) return TTS_ENGINE_RESIDENT;
    return -1;
}

int engine_create(const tts_system_desc &d, const std::vector<HostInstance> &host,
                  const std::vector<std::vector<int64_t>> &slot_of_atom, const std::vector<DevInstance> &dinst,
                  const StepParams &p, const DevBuffers &b, int engine, cudaStream_t st, EngineState **out)
{
    (void)slot_of_atom;
    (void)p;
    *out = nullptr;
    EngineState *e = new EngineState;
    e->engine = engine;
    e->precision = d.precision;
    e->n_inst = static_cast<int>(host.size());
    e->dinst = dinst;
    for (const DevInstance &di : dinst) e->n_total += di.n;
    fill_species<float>(d, e->spf);
    fill_species<double>(d, e->spd);
    cudaError_t ce;
    if (engine == TTS_ENGINE_CHECKER) {
        std::vector<CheckerInst> ci(e->n_inst);
        int64_t prefix = 0;
        for (int i = 0; i < e->n_inst; ++i) {
            const HostInstance &hi = host[i];
            CheckerInst &c = ci[i];
            c.slot_begin = dinst[i].slot_begin;
            c.prefix = prefix;
            c.nhalf = static_cast<uint32_t>(hi.n / 2);
            c.Lx = hi.cells[0];
            c.Ly = hi.cells[1];
            c.Lz = hi.cells[2];
            c.hx = c.Lx / 2;
            c.inst_global = static_cast<uint32_t>(d.instance_base + i);
            c.div_hx = make_fastdiv(c.hx);
            c.div_Ly = make_fastdiv(c.Ly);
            if (hi.ncolours != 2 || dinst[i].colour_begin[1] != int64_t(c.nhalf)) {
                delete e;
                return eng_fail(TTS_ERR_UNSUPPORTED, "checker engine needs the parity colouring");
            }
            // the kernel's index arithmetic relies on these divisions being exact
            if (!fastdiv_ok(c.hx, c.nhalf) || !fastdiv_ok(c.Ly, c.Ly * c.Lz)) {
                delete e;
                return eng_fail(TTS_ERR_UNSUPPORTED, "fast division check failed");
            }
            prefix += c.nhalf;
        }
        e->work = prefix;
        const size_t vs = d.precision == 64 ? sizeof(double4a) : sizeof(float4);
        if ((ce = cudaMalloc(&e->S, size_t(e->n_total) * vs)) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->ci), ci.size() * sizeof(CheckerInst))) != cudaSuccess) {
            cudaGetLastError();
            engine_destroy(e);
            return eng_fail(TTS_ERR_OOM, std::string("checker buffers: ") + cudaGetErrorString(ce));
        }
        cudaMemcpyAsync(e->ci, ci.data(), ci.size() * sizeof(CheckerInst), cudaMemcpyHostToDevice, st);
        if ((ce = engine_sync_from_general(e, b, st)) != cudaSuccess || (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
            engine_destroy(e);
            return eng_fail(TTS_ERR_CUDA, std::string("checker set-up: ") + cudaGetErrorString(ce));
        }
    } else if (engine == TTS_ENGINE_RESIDENT) {
        std::vector<ResInst> ri(e->n_inst);
        std::vector<int> order(e->n_inst);
        for (int i = 0; i < e->n_inst; ++i) {
            const HostInstance &hi = host[i];
            ResInst &r = ri[i];
            std::memset(&r, 0, sizeof r);
            r.slot_begin = dinst[i].slot_begin;
            r.n = static_cast<int>(hi.n);
            for (int k = 0; k < 3; ++k) r.L[k] = hi.cells[k];
            r.divx = make_fastdiv(hi.cells[0]);
            r.divxy = make_fastdiv(hi.cells[0] * hi.cells[1]);
            if (!fastdiv_ok(hi.cells[0], hi.cells[0] * hi.cells[1]) ||
                !fastdiv_ok(hi.cells[0] * hi.cells[1], static_cast<uint32_t>(hi.n))) {
                delete e;
                return eng_fail(TTS_ERR_UNSUPPORTED, "fast division check failed");
            }
            for (int c = 0; c <= hi.ncolours; ++c) r.colour_begin[c] = static_cast<int>(dinst[i].colour_begin[c]);
            r.ncolours = hi.ncolours;
            r.inst = i;
            r.inst_global = static_cast<uint32_t>(d.instance_base + i);
            e->nmax = std::max(e->nmax, r.n);
            order[i] = i;
        }
        // largest instances first (longest-processing-time order)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ri[x].n > ri[y].n; });
        e->smem = resident_bytes(e->nmax, d.precision);
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        e->block = 512;
        cudaError_t a1 = d.precision == 64
                             ? cudaFuncSetAttribute(resident_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(e->smem))
                             : cudaFuncSetAttribute(resident_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(e->smem));
        int per_sm = 0;
        if (a1 == cudaSuccess)
            a1 = d.precision == 64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel<double>,
                                                                                  e->block, e->smem)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel<float>,
                                                                                  e->block, e->smem);
        if (a1 != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            delete e;
            return eng_fail(TTS_ERR_UNSUPPORTED, "resident kernel does not fit one CTA per SM");
        }
        e->grid = std::min(e->n_inst, nsm * per_sm);
        if ((ce = cudaMalloc(reinterpret_cast<void **>(&e->ri), ri.size() * sizeof(ResInst))) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->order), order.size() * sizeof(int))) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->queue), sizeof(int))) != cudaSuccess) {
            cudaGetLastError();
            engine_destroy(e);
            return eng_fail(TTS_ERR_OOM, std::string("resident buffers: ") + cudaGetErrorString(ce));
        }
        cudaMemcpyAsync(e->ri, ri.data(), ri.size() * sizeof(ResInst), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(e->order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(e->queue, 0, sizeof(int), st);
        if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) {
            engine_destroy(e);
            return eng_fail(TTS_ERR_CUDA, std::string("resident set-up: ") + cudaGetErrorString(ce));
        }
    } else {
        delete e;
        return eng_fail(TTS_ERR_UNSUPPORTED, "unknown engine");
    }
    *out = e;
    return TTS_OK;
}

void engine_destroy(EngineState *e)
{
    if (!e) return;
    for (void *q : {e->S, static_cast<void *>(e->ci), static_cast<void *>(e->ri), static_cast<void *>(e->order),
                    static_cast<void *>(e->queue)})
        if (q) cudaFree(q);
    delete e;
}

bool engine_multi_step(const EngineState *e) { return e && e->engine == TTS_ENGINE_RESIDENT; }

cudaError_t engine_record_step(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                               bool ttm_active, cudaStream_t st, int *kernels, cudaEvent_t ev0, cudaEvent_t ev1)
{
    *kernels = 0;
    if (e->engine != TTS_ENGINE_CHECKER) return cudaErrorNotSupported;
    cudaError_t err = launch_sigma(p, b, p.ncells_total, e->precision, st);
    ++*kernels;
    if (err == cudaSuccess && ev0) err = cudaEventRecord(ev0, st);
    const int npass = 2 * e->K - 1;
    for (int pass = 0; pass < npass && err == cudaSuccess; ++pass) {
        const int c = pass < e->K - 1 ? pass : (pass == e->K - 1 ? e->K - 1 : 2 * e->K - 2 - pass);
        const int hsel = pass == e->K - 1 ? 1 : 0;
        const int bs = 256;
        const int64_t gs = (e->work + bs - 1) / bs;
        if (e->precision == 64) {
            CheckerArgs<double> a{};
            a.S = static_cast<double4a *>(e->S);
            a.ci = e->ci;
            a.cell = b.cell;
            a.sigma = static_cast<const double *>(b.sigma);
            a.step = b.step;
            a.health = b.health;
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spd[t];
            a.nx = p.axis[0]; a.ny = p.axis[1]; a.nz = p.axis[2];
            a.Bx = p.B[0]; a.By = p.B[1]; a.Bz = p.B[2];
            a.dt = p.dt;
            a.key0 = p.key0; a.key1 = p.key1;
            a.n_inst = e->n_inst;
            a.total = e->work;
            checker_pass_kernel<double><<<gs, bs, 0, st>>>(a, c, hsel, pass);
        } else {
            CheckerArgs<float> a{};
            a.S = static_cast<float4 *>(e->S);
            a.ci = e->ci;
            a.cell = b.cell;
            a.sigma = static_cast<const float *>(b.sigma);
            a.step = b.step;
            a.health = b.health;
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spf[t];
            a.nx = float(p.axis[0]); a.ny = float(p.axis[1]); a.nz = float(p.axis[2]);
            a.Bx = float(p.B[0]); a.By = float(p.B[1]); a.Bz = float(p.B[2]);
            a.dt = float(p.dt);
            a.key0 = p.key0; a.key1 = p.key1;
            a.n_inst = e->n_inst;
            a.total = e->work;
            checker_pass_kernel<float><<<gs, bs, 0, st>>>(a, c, hsel, pass);
        }
        err = cudaGetLastError();
        ++*kernels;
    }
    if (err == cudaSuccess && ev1) err = cudaEventRecord(ev1, st);
    if (err == cudaSuccess && ttm_active) {
        err = launch_ttm(p, b, tp, p.n_instances, st);
        ++*kernels;
    }
    if (err == cudaSuccess && p.sample_every > 0) {
        const int bs = 256;
        const int64_t gs = (e->n_total + bs - 1) / bs;
        if (e->precision == 64)
            to_general_kernel<double><<<gs, bs, 0, st>>>(static_cast<const double4a *>(e->S), static_cast<double *>(b.sx),
                                                         static_cast<double *>(b.sy), static_cast<double *>(b.sz),
                                                         e->n_total, b.step, p.sample_every, 1);
        else
            to_general_kernel<float><<<gs, bs, 0, st>>>(static_cast<const float4 *>(e->S), static_cast<float *>(b.sx),
                                                        static_cast<float *>(b.sy), static_cast<float *>(b.sz),
                                                        e->n_total, b.step, p.sample_every, 1);
        err = cudaGetLastError();
        ++*kernels;
    }
    if (err == cudaSuccess) {
        err = launch_obs(p, b, e->precision, p.obs_blocks, 0, st);
        *kernels += 2;
    }
    return err;
}

cudaError_t engine_run_steps(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                             bool ttm_active, int64_t nsteps, cudaStream_t st, int *kernels, cudaEvent_t ev0,
                             cudaEvent_t ev1)
{
    *kernels = 0;
    if (e->engine != TTS_ENGINE_RESIDENT) return cudaErrorNotSupported;
    cudaError_t err = cudaSuccess;
    if (ev0) err = cudaEventRecord(ev0, st);
    auto fill = [&](auto &a) {
        a.species = b.species;
        a.atom = b.atom;
        a.ri = e->ri;
        a.order = e->order;
        a.queue = e->queue;
        a.step = b.step;
        a.health = b.health;
        a.Te = b.Te;
        a.Tl = b.Tl;
        a.src_energy = b.src_energy;
        a.inst = b.inst;
        a.obs_ring = b.obs_ring;
        a.obs_count = b.obs_count;
        for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.spd[t] = p.sp[t];
        for (int k = 0; k < 3; ++k) {
            a.axis[k] = p.axis[k];
            a.B[k] = p.B[k];
        }
        a.dt = p.dt;
        a.key0 = p.key0;
        a.key1 = p.key1;
        a.n_inst = e->n_inst;
        a.nspecies = p.nspecies;
        a.sample_every = p.sample_every;
        a.obs_capacity = p.obs_capacity;
        a.nmax = e->nmax;
        a.ttm_active = ttm_active ? 1 : 0;
        a.tp = tp;
    };
    if (err == cudaSuccess) {
        if (e->precision == 64) {
            ResArgs<double> a{};
            a.sx = static_cast<double *>(b.sx);
            a.sy = static_cast<double *>(b.sy);
            a.sz = static_cast<double *>(b.sz);
            fill(a);
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spd[t];
            resident_kernel<double><<<e->grid, e->block, e->smem, st>>>(a, nsteps);
        } else {
            ResArgs<float> a{};
            a.sx = static_cast<float *>(b.sx);
            a.sy = static_cast<float *>(b.sy);
            a.sz = static_cast<float *>(b.sz);
            fill(a);
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spf[t];
            resident_kernel<float><<<e->grid, e->block, e->smem, st>>>(a, nsteps);
        }
        err = cudaGetLastError();
        ++*kernels;
    }
    if (err == cudaSuccess && ev1) err = cudaEventRecord(ev1, st);
    if (err == cudaSuccess) {
        advance_step_kernel<<<1, 1, 0, st>>>(b.step, nsteps, e->queue);
        err = cudaGetLastError();
        ++*kernels;
    }
    return err;
}

int engine_set_cells(EngineState *e, const std::vector<DevInstance> &dinst, const std::vector<int> &, cudaStream_t)
{
    e->dinst = dinst;
    if (e->engine == TTS_ENGINE_RESIDENT)
        for (const DevInstance &di : dinst)
            if (di.ncells != 1) return eng_fail(TTS_ERR_UNSUPPORTED, "the resident engine takes one TTM cell per instance");
    return TTS_OK;
}

cudaError_t engine_sync_to_general(EngineState *e, const DevBuffers &b, cudaStream_t st)
{
    if (e->engine != TTS_ENGINE_CHECKER) return cudaSuccess;
    const int bs = 256;
    const int64_t gs = (e->n_total + bs - 1) / bs;
    if (e->precision == 64)
        to_general_kernel<double><<<gs, bs, 0, st>>>(static_cast<const double4a *>(e->S), static_cast<double *>(b.sx),
                                                     static_cast<double *>(b.sy), static_cast<double *>(b.sz),
                                                     e->n_total, b.step, 0, 0);
    else
        to_general_kernel<float><<<gs, bs, 0, st>>>(static_cast<const float4 *>(e->S), static_cast<float *>(b.sx),
                                                    static_cast<float *>(b.sy), static_cast<float *>(b.sz), e->n_total,
                                                    b.step, 0, 0);
    return cudaGetLastError();
}

cudaError_t engine_sync_from_general(EngineState *e, const DevBuffers &b, cudaStream_t st)
{
    if (e->engine != TTS_ENGINE_CHECKER) return cudaSuccess;
    const int bs = 256;
    const int64_t gs = (e->n_total + bs - 1) / bs;
    if (e->precision == 64)
        from_general_kernel<double><<<gs, bs, 0, st>>>(static_cast<double4a *>(e->S), static_cast<const double *>(b.sx),
                                                       static_cast<const double *>(b.sy),
                                                       static_cast<const double *>(b.sz), b.species, e->n_total);
    else
        from_general_kernel<float><<<gs, bs, 0, st>>>(static_cast<float4 *>(e->S), static_cast<const float *>(b.sx),
                                                      static_cast<const float *>(b.sy), static_cast<const float *>(b.sz),
                                                      b.species, e->n_total);
    return cudaGetLastError();
}

}  // namespace tts
