// tts_kernels.cu -- device kernels of the general engine.
//
//  sigma      noise amplitude table sqrt(2 alpha k_B T_e / (gamma mu h)) per
//             (TTM cell, species, h) from the FP64 electron temperature
//             (paper Eq. 2 with the FDT 1/sqrt(mu) scaling of Sec. II.C)
//  pass       one colour class advanced by h: exchange/anisotropy/Zeeman field
//             scaled by 1/mu (Sec. II.C), Philox noise, exact frozen-field
//             LLG flow (Eq. 1), renormalisation
//  ttm        FP64 two-temperature-model grid advance (fix ttm, Sec. II.B)
//  obs        FP64 per-instance reductions of magnetisation, energies and
//             spin temperatures, reduced in a fixed order (deterministic)
#include <cmath>

#include "tts_kernels.h"
#include "tts_philox.cuh"

namespace tts {
namespace {

template <typename R>
struct Math;

template <>
struct Math<float> {
    static constexpr float tiny = 1e-30f;
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float exp_(float x) { return expf(x); }
    __device__ static float log_(float x) { return logf(x); }
    __device__ static void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    __device__ static void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
    __device__ static float uniform(uint32_t w) { return uniform_f(w); }
};

template <>
struct Math<double> {
    static constexpr double tiny = 1e-300;
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double exp_(double x) { return exp(x); }
    __device__ static double log_(double x) { return log(x); }
    __device__ static void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
    __device__ static void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
    __device__ static double uniform(uint32_t w) { return uniform_d(w); }
};

// Three standard normals from one Philox block by Box-Muller:
// g1, g2 = sqrt(-2 ln u0) (cos, sin)(2 pi u1), g3 = sqrt(-2 ln u2) cos(2 pi u3).
template <typename R>
__device__ __forceinline__ void gauss3(const u32x4 &w, R &g1, R &g2, R &g3)
{
    using M = Math<R>;
    const R u0 = M::uniform(w.x), u1 = M::uniform(w.y), u2 = M::uniform(w.z), u3 = M::uniform(w.w);
    const R r01 = M::sqrt_(R(-2) * M::log_(u0));
    const R r23 = M::sqrt_(R(-2) * M::log_(u2));
    R s1, c1, s3, c3;
    M::sincospi_(R(2) * u1, &s1, &c1);
    M::sincospi_(R(2) * u3, &s3, &c3);
    g1 = r01 * c1;
    g2 = r01 * s1;
    g3 = r23 * c3;
}

// Exact solution of Eq. 1 for one spin in a field held fixed for time h:
// precession about b = B/|B| at w = gamma' |B| (counter-clockwise) and the
// polar half-angle tangent relaxing as tan(theta/2) -> tan(theta/2) e^{-alpha w h}.
template <typename R>
__device__ __forceinline__ void exact_flow(R &sx, R &sy, R &sz, R Bx, R By, R Bz, R alpha, R gprime, R h)
{
    using M = Math<R>;
    const R B2 = Bx * Bx + By * By + Bz * Bz;
    if (!(B2 > R(0))) return;
    const R Bm = M::sqrt_(B2);
    const R ib = R(1) / Bm;
    const R bx = Bx * ib, by = By * ib, bz = Bz * ib;
    const R c = sx * bx + sy * by + sz * bz;
    const R px = sx - c * bx, py = sy - c * by, pz = sz - c * bz;
    const R pm = M::sqrt_(px * px + py * py + pz * pz);
    if (pm <= Math<R>::tiny) return;
    const R ip = R(1) / pm;
    const R e1x = px * ip, e1y = py * ip, e1z = pz * ip;
    const R e2x = by * e1z - bz * e1y;
    const R e2y = bz * e1x - bx * e1z;
    const R e2z = bx * e1y - by * e1x;
    const R u0 = (c >= R(0)) ? pm / (R(1) + c) : (R(1) - c) / pm;
    const R w = gprime * Bm;
    const R u = u0 * M::exp_(-alpha * w * h);
    const R u2 = u * u;
    const R inv = R(1) / (R(1) + u2);
    const R cn = (R(1) - u2) * inv;
    const R sn = R(2) * u * inv;
    R sp, cp;
    M::sincos_(w * h, &sp, &cp);
    R ox = cn * bx + sn * (cp * e1x + sp * e2x);
    R oy = cn * by + sn * (cp * e1y + sp * e2y);
    R oz = cn * bz + sn * (cp * e1z + sp * e2z);
    const R on = R(1) / M::sqrt_(ox * ox + oy * oy + oz * oz);
    sx = ox * on;
    sy = oy * on;
    sz = oz * on;
}

// ---------------------------------------------------------------------------
// Noise amplitude sqrt(2 alpha k_B T / (gamma mu h)) of one cell, written for
// both species and both sub-step lengths (h = dt/2, dt).  One formula for
// every kernel that refreshes the table, so a restart reproduces a
// continuous run bit for bit.
template <typename R>
__device__ __forceinline__ void write_sigma(const StepParams &p, double T, R *__restrict__ sigma, int64_t g)
{
    // sigma = sqrt(2 alpha k_B T / (gamma mu h)) (paper Eq. 2) as sqrt(T) times
    // the per-species, per-h factor
    const double rT = T > 0.0 ? sqrt(T) : 0.0;
    for (int t = 0; t < TTS_MAX_SPECIES; ++t)
        for (int hs = 0; hs < 2; ++hs) {
            const double v = t < p.nspecies ? p.sp[t].sig_c[hs] * rT : 0.0;
            sigma[(g * TTS_MAX_SPECIES + t) * 2 + hs] = static_cast<R>(v);
        }
}

template <typename R>
__global__ void sigma_kernel(StepParams p, const double *__restrict__ Te, R *__restrict__ sigma, int ncells)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncells) return;
    write_sigma<R>(p, Te[g], sigma, g);
}

// Field of one slot from the neighbour table (J/mu already folded in), the
// anisotropy and the applied field.
template <typename R>
__device__ __forceinline__ void det_field(const StepParams &p, int64_t slot, int t, R sx, R sy, R sz,
                                          const R *__restrict__ S0, const R *__restrict__ S1,
                                          const R *__restrict__ S2, const int *__restrict__ nbr,
                                          const R *__restrict__ w, R &Bx, R &By, R &Bz)
{
    R hx = 0, hy = 0, hz = 0;
    for (int k = 0; k < p.zmax; ++k) {
        const int64_t e = int64_t(k) * p.n_total + slot;
        const R J = w[e];
        const int j = nbr[e];
        hx += J * S0[j];
        hy += J * S1[j];
        hz += J * S2[j];
    }
    const R nx = R(p.axis[0]), ny = R(p.axis[1]), nz = R(p.axis[2]);
    const R sn = sx * nx + sy * ny + sz * nz;
    const R ka = R(p.sp[t].kappa) * sn;
    Bx = hx + ka * nx + R(p.B[0]);
    By = hy + ka * ny + R(p.B[1]);
    Bz = hz + ka * nz + R(p.B[2]);
}

template <typename R>
__global__ void __launch_bounds__(512) pass_general_kernel(StepParams p, DevBuffers b, int pass,
                                                           const PassRange *__restrict__ ranges, int nranges,
                                                           int64_t nwork, SweepCtl sw)
{
    int hsel_dyn = -1;
    if (sw.mode != 0 && !sweep_gate(sw, b.step, hsel_dyn)) return;
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= nwork) return;
    int lo = 0, hi = nranges - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ranges[mid].prefix <= gid) lo = mid; else hi = mid - 1;
    }
    const PassRange r = ranges[lo];
    const int64_t slot = r.slot_begin + (gid - r.prefix);
    R *S0 = static_cast<R *>(b.sx), *S1 = static_cast<R *>(b.sy), *S2 = static_cast<R *>(b.sz);
    const int t = b.species[slot];
    R sx = S0[slot], sy = S1[slot], sz = S2[slot];
    R Bx, By, Bz;
    det_field<R>(p, slot, t, sx, sy, sz, S0, S1, S2, b.nbr, static_cast<const R *>(b.nbr_w), Bx, By, Bz);
    const int hsel = hsel_dyn >= 0 ? hsel_dyn : r.hsel;
    const R h = hsel ? R(p.dt) : R(0.5 * p.dt);
    const R sig = static_cast<const R *>(b.sigma)[(int64_t(b.cell[slot]) * TTS_MAX_SPECIES + t) * 2 + hsel];
    if (sig > R(0)) {
        const int64_t step = *b.step;
        u32x4 c{static_cast<uint32_t>(b.atom[slot]), static_cast<uint32_t>(step), static_cast<uint32_t>(pass),
                static_cast<uint32_t>(p.instance_base + r.inst)};
        const u32x4 wv = philox4x32_10(c, p.key0, p.key1);
        R g1, g2, g3;
        gauss3<R>(wv, g1, g2, g3);
        Bx += sig * g1;
        By += sig * g2;
        Bz += sig * g3;
    }
    // on-site anisotropy at the predicted sub-step midpoint:
    // B += kappa (h/2) dc/dt n, dc/dt = -gamma' [n.(s x B) + alpha (c s.B - n.B)]
    const R alpha = R(p.sp[t].alpha), gp = R(p.sp[t].gprime), kap = R(p.sp[t].kappa);
    if (kap != R(0)) {
        const R nx = R(p.axis[0]), ny = R(p.axis[1]), nz = R(p.axis[2]);
        const R c = sx * nx + sy * ny + sz * nz;
        const R cx = sy * Bz - sz * By, cy = sz * Bx - sx * Bz, cz = sx * By - sy * Bx;
        const R n_sxB = nx * cx + ny * cy + nz * cz;
        const R sB = sx * Bx + sy * By + sz * Bz;
        const R nB = nx * Bx + ny * By + nz * Bz;
        const R cdot = -gp * (n_sxB + alpha * (c * sB - nB));
        const R corr = kap * R(0.5) * h * cdot;
        Bx += corr * nx;
        By += corr * ny;
        Bz += corr * nz;
    }
    exact_flow<R>(sx, sy, sz, Bx, By, Bz, alpha, gp, h);
    if (!(isfinite(sx) && isfinite(sy) && isfinite(sz))) atomicOr(b.health, kHealthNonFinite);
    S0[slot] = sx;
    S1[slot] = sy;
    S2[slot] = sz;
}

// ---------------------------------------------------------------------------
// TTM: one block per instance, cells strided over the block, FP64.
// ---------------------------------------------------------------------------
__global__ void ttm_kernel(StepParams p, DevBuffers b, TtmParams tp)
{
    const DevInstance I = b.inst[blockIdx.x];
    const int nc = I.ncells;
    double *Te = b.Te + I.cell_begin, *Tl = b.Tl + I.cell_begin;
    double *dE = b.ttm_scratch + I.cell_begin;   // electron-energy increments of one sub-step
    const double *shape = b.src_shape + I.cell_begin;
    const int64_t step = *b.step;
    const double delta = p.dt / I.substeps;
    double deposited = 0.0;
    const int nxc = I.cells[0], nyc = I.cells[1], nzc = I.cells[2];
    for (int k = 0; k < I.substeps; ++k) {
        const double t = double(step) * p.dt + double(k) * delta;
        double pulse = 0.0;
        if (tp.source != TTS_SOURCE_NONE) {
            const double z = (t - I.t0) / I.sigma_t;
            pulse = I.P0 * exp(-0.5 * z * z);
        }
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const int cx = c % nxc, cy = (c / nxc) % nyc, cz = c / (nxc * nyc);
            const double Tc = Te[c];
            double lap = 0.0;
            if (nxc > 1) {
                const double a = Te[cz * nyc * nxc + cy * nxc + (cx + 1) % nxc];
                const double m = Te[cz * nyc * nxc + cy * nxc + (cx + nxc - 1) % nxc];
                lap += (a - 2.0 * Tc + m) / (I.dx[0] * I.dx[0]);
            }
            if (nyc > 1) {
                const double a = Te[cz * nyc * nxc + ((cy + 1) % nyc) * nxc + cx];
                const double m = Te[cz * nyc * nxc + ((cy + nyc - 1) % nyc) * nxc + cx];
                lap += (a - 2.0 * Tc + m) / (I.dx[1] * I.dx[1]);
            }
            if (nzc > 1) {
                const double a = Te[((cz + 1) % nzc) * nyc * nxc + cy * nxc + cx];
                const double m = Te[((cz + nzc - 1) % nzc) * nyc * nxc + cy * nxc + cx];
                lap += (a - 2.0 * Tc + m) / (I.dx[2] * I.dx[2]);
            }
            const double src = pulse * shape[c];
            const double x = tp.G * (Tc - Tl[c]);
            dE[c] = delta * (tp.kappa_e * lap - x + src);
            deposited += delta * src * I.cell_volume;
            // T_l of a cell is read by that cell's thread only: update in place
            Tl[c] += delta * x / tp.C_l;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const double Ee = 0.5 * tp.gamma_e * Te[c] * Te[c] + dE[c];
            Te[c] = sqrt(2.0 * Ee / tp.gamma_e);
        }
        __syncthreads();
    }
    // fixed-order block reduction of the deposited energy
    __shared__ double red[256];
    red[threadIdx.x] = deposited;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) b.src_energy[blockIdx.x] += red[0];
}

// ---------------------------------------------------------------------------
// TTM with one sub-step per spin step (the usual case): the electron-energy
// increments of all cells of all instances in one grid, then the update per
// instance.
// ---------------------------------------------------------------------------
__global__ void ttm_increment_kernel(StepParams p, DevBuffers b, TtmParams tp, const int *__restrict__ cell_inst,
                                     int ncells_total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncells_total) return;
    const int inst = cell_inst[g];
    const DevInstance &I = b.inst[inst];
    const int c = g - I.cell_begin;
    const double *Te = b.Te + I.cell_begin;
    const int nxc = I.cells[0], nyc = I.cells[1], nzc = I.cells[2];
    const int cx = c % nxc, cy = (c / nxc) % nyc, cz = c / (nxc * nyc);
    const double Tc = Te[c];
    double lap = 0.0;
    if (nxc > 1)
        lap += (Te[cz * nyc * nxc + cy * nxc + (cx + 1) % nxc] - 2.0 * Tc + Te[cz * nyc * nxc + cy * nxc + (cx + nxc - 1) % nxc]) *
               I.inv_dx2[0];
    if (nyc > 1)
        lap += (Te[cz * nyc * nxc + ((cy + 1) % nyc) * nxc + cx] - 2.0 * Tc + Te[cz * nyc * nxc + ((cy + nyc - 1) % nyc) * nxc + cx]) *
               I.inv_dx2[1];
    if (nzc > 1)
        lap += (Te[((cz + 1) % nzc) * nyc * nxc + cy * nxc + cx] - 2.0 * Tc +
                Te[((cz + nzc - 1) % nzc) * nyc * nxc + cy * nxc + cx]) * I.inv_dx2[2];
    double pulse = 0.0;
    if (tp.source != TTS_SOURCE_NONE) {
        const double z = (double(*b.step) * p.dt - I.t0) / I.sigma_t;
        pulse = I.P0 * exp(-0.5 * z * z);
    }
    const double src = pulse * b.src_shape[g];
    const double x = tp.G * (Tc - b.Tl[g]);
    b.ttm_scratch[g] = p.dt * (tp.kappa_e * lap - x + src);
    b.Tl[g] += p.dt * x * tp.inv_C_l;
}

// New T_e of every cell and, from it, the noise table of the next step; the
// step counter advances here when no observable kernel follows.
template <typename R>
__global__ void ttm_apply_kernel(StepParams p, DevBuffers b, TtmParams tp, int ncells_total, int inc_step)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    // the table of the next step: sigma, or with sigma_alternate the one of
    // that step's parity (the colour passes of this step may still read the
    // other; the step counter is advanced after them)
    R *out = static_cast<R *>(p.sigma_alternate && !p.sigma_parity ? b.sigma_alt : b.sigma);
    if (inc_step && !p.sigma_alternate && g == 0) *b.step += 1;
    if (g >= ncells_total) return;
    // electron energy gamma_e T^2 / 2 plus the increment, back to T
    const double T0 = b.Te[g];
    const double T = sqrt(fma(2.0 * b.ttm_scratch[g], tp.inv_gamma_e, T0 * T0));
    b.Te[g] = T;
    write_sigma<R>(p, T, out, g);
}

// Prescribed three-stage T_e (step profile) at time t.
__device__ __forceinline__ double profile_Te(const DevInstance &I, double t, double T_base)
{
    return t < I.prof_t1 ? I.prof_peak : (t < I.prof_t2 ? 0.5 * I.prof_peak : T_base);
}

// Step profile: T_e of every cell at t_n+1 and the noise table of the next
// step from it; T_l stays at the base temperature.
template <typename R>
__global__ void ttm_profile_kernel(StepParams p, DevBuffers b, TtmParams tp, const int *__restrict__ cell_inst,
                                   int ncells_total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncells_total) return;
    const DevInstance &I = b.inst[cell_inst[g]];
    const double T = profile_Te(I, double(*b.step + 1) * p.dt, tp.T0);
    b.Te[g] = T;
    b.Tl[g] = tp.T0;
    write_sigma<R>(p, T, static_cast<R *>(b.sigma), g);
}

// ---------------------------------------------------------------------------
// Observables.  mode 0: inside a step (sample when (step+1) % every == 0, into
// the ring, then advance the step counter); mode 1: now, into obs_now.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kObsBlock) obs_partial_kernel(StepParams p, DevBuffers b, int mode)
{
    const int64_t step = *b.step;
    const int64_t clock = p.lattice_on ? *p.lstep : step;
    if (mode == 0 && (p.sample_every <= 0 || (clock + 1) % p.sample_every != 0)) return;
    const R *S0 = static_cast<const R *>(b.sx), *S1 = static_cast<const R *>(b.sy), *S2 = static_cast<const R *>(b.sz);
    const R *w = static_cast<const R *>(b.nbr_w);
    // a small persistent grid walks the observable blocks, so steps that do
    // not sample cost one early exit per CTA
    for (int blk = blockIdx.x; blk < p.obs_blocks; blk += gridDim.x) {
        const int inst = b.obs_block_inst[blk];
        const DevInstance I = b.inst[inst];
        const int64_t first = b.obs_block_begin[blk];
        const int64_t end = I.slot_begin + I.n;
        double acc[kObsFields];
#pragma unroll
        for (int k = 0; k < kObsFields; ++k) acc[k] = 0.0;
        for (int j = 0; j < kObsSpan / kObsBlock; ++j) {
            const int64_t slot = first + threadIdx.x + int64_t(j) * kObsBlock;
            if (slot >= end) break;
            const int t = b.species[slot];
            const double sx = S0[slot], sy = S1[slot], sz = S2[slot];
            double hx = 0, hy = 0, hz = 0;
            for (int k = 0; k < p.zmax; ++k) {
                const int64_t e = int64_t(k) * p.n_total + slot;
                const double J = w[e];
                const int jn = b.nbr[e];
                hx += J * double(S0[jn]);
                hy += J * double(S1[jn]);
                hz += J * double(S2[jn]);
            }
            const double mu = p.sp[t].mu;
            const double sn = sx * p.axis[0] + sy * p.axis[1] + sz * p.axis[2];
            const double ka = p.sp[t].kappa * sn;
            const double Bx = hx + ka * p.axis[0] + p.B[0];
            const double By = hy + ka * p.axis[1] + p.B[1];
            const double Bz = hz + ka * p.axis[2] + p.B[2];
            const double Hx = mu * Bx, Hy = mu * By, Hz = mu * Bz;
            const double cx = sy * Hz - sz * Hy, cy = sz * Hx - sx * Hz, cz = sx * Hy - sy * Hx;
            const double v[12] = {1.0, sx, sy, sz, 0.0, 0.0, 0.0,
                                  -0.5 * mu * (sx * hx + sy * hy + sz * hz),
                                  -p.sp[t].K * sn * sn,
                                  -mu * (p.B[0] * sx + p.B[1] * sy + p.B[2] * sz),
                                  cx * cx + cy * cy + cz * cz,
                                  sx * Hx + sy * Hy + sz * Hz};
            // species select without indexing the accumulator by t
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[k] += t == 0 ? v[k] : 0.0;
                acc[12 + k] += t == 0 ? 0.0 : v[k];
            }
        }
        block_sum_store<kObsFields>(acc, b.obs_partial + int64_t(blk) * kObsFields);
    }
}

// Per species t the partial sums are, at 12 t + k: k = 0 count, 1..3 sum s,
// 4..6 unused, 7 exchange energy (half of mu s.h per atom, each pair counted
// twice), 8 anisotropy, 9 Zeeman, 10 sum |s x H|^2, 11 sum s.H.  The moment-
// weighted direction is sum_t mu_t sum_{i in t} s_i / sum_t mu_t n_t.
constexpr int kObsReduceThreads = 32 * (kObsFields + 4);   // one warp a field

__global__ void __launch_bounds__(kObsReduceThreads) obs_reduce_kernel(StepParams p, DevBuffers b, int mode)
{
    const int64_t step = *b.step;
    const int64_t clock = p.lattice_on ? *p.lstep : step;
    const bool sample = (mode == 1) || (p.sample_every > 0 && (clock + 1) % p.sample_every == 0);
    if (!sample) return;
    const int inst = blockIdx.x;
    const DevInstance I = b.inst[inst];
    // warp f sums field f in a fixed order: lane j the blocks j, j + 32, ...
    // (TTM cells and lattice partials likewise), then a shuffle tree.  Extra
    // fields: sum T_e, sum T_l, kinetic and pair energy.  One warp a field
    // spreads the FP64 adds over the SM's four schedulers.
    constexpr int NF = kObsFields + 4;
    __shared__ double red[NF];
    const int lane = threadIdx.x & 31, f = threadIdx.x >> 5;
    double part = 0.0;
    const int blk_end = I.obs_block_begin + I.obs_block_count;
    if (f < kObsFields) {
        for (int blk = I.obs_block_begin + lane; blk < blk_end; blk += 32)
            part += b.obs_partial[int64_t(blk) * kObsFields + f];
    } else if (f < kObsFields + 2) {
        const double *T = f == kObsFields ? b.Te : b.Tl;
        for (int c = lane; c < I.ncells; c += 32) part += T[I.cell_begin + c];
    } else if (f < NF && p.lattice_on && mode == 0) {
        for (int blk = I.obs_block_begin + lane; blk < blk_end; blk += 32)
            part += p.lat_partial[2 * int64_t(blk) + (f - kObsFields - 2)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if (lane == 0 && f < NF) red[f] = part;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[kObsFields];
    for (int k = 0; k < kObsFields; ++k) tot[k] = red[k];
    double rec[TTS_NOBS];
    for (int k = 0; k < TTS_NOBS; ++k) rec[k] = 0.0;
    // a moving lattice has advanced the spin-step counter already
    const int64_t sstep = (mode == 0 && !p.lattice_on) ? step + 1 : step;
    rec[0] = double(sstep) * p.dt;
    double musum = 0.0, mux = 0.0, muy = 0.0, muz = 0.0;
    for (int t = 0; t < TTS_MAX_SPECIES; ++t) {
        const double *a = tot + 12 * t;
        const double cnt = a[0];
        if (cnt > 0.0) {
            rec[1 + 3 * t] = a[1] / cnt;
            rec[2 + 3 * t] = a[2] / cnt;
            rec[3 + 3 * t] = a[3] / cnt;
            const double m = p.sp[t].mu / kBohrMagneton;
            musum += m * cnt;
            mux += m * a[1];
            muy += m * a[2];
            muz += m * a[3];
        }
        rec[10] += a[7];
        rec[11] += a[8];
        rec[12] += a[9];
        rec[13 + t] = (cnt > 0.0 && a[11] != 0.0) ? a[10] / (2.0 * kBoltzmann * a[11]) : 0.0;
    }
    rec[7] = mux / musum;
    rec[8] = muy / musum;
    rec[9] = muz / musum;
    rec[15] = red[kObsFields] / I.ncells;
    rec[16] = red[kObsFields + 1] / I.ncells;
    if (p.lattice_on && mode == 0) {
        const double ek = red[kObsFields + 2], em = red[kObsFields + 3];
        rec[16] = 2.0 * ek / (3.0 * double(I.n) * kBoltzmann);
        rec[17] = ek;
        rec[18] = em;
    }
    rec[19] = double(sstep);
    double *dst;
    if (mode == 0) {
        const int64_t k = b.obs_count[inst];
        dst = b.obs_ring + (int64_t(inst) * p.obs_capacity + (k % p.obs_capacity)) * TTS_NOBS;
        b.obs_count[inst] = k + 1;
    } else {
        dst = b.obs_now + int64_t(inst) * TTS_NOBS;
    }
    for (int k = 0; k < TTS_NOBS; ++k) dst[k] = rec[k];
}

__global__ void step_inc_kernel(int64_t *step) { *step += 1; }

// ---------------------------------------------------------------------------
// Source calibration.  The TTM-only run uses the same update as ttm_kernel;
// every thread keeps the running maximum of its cells and the block reduces
// it once per run.
// ---------------------------------------------------------------------------
__device__ double calib_peak(const CalibJob &J, double P0, double dt, const TtmParams &tp, double *work, double *red)
{
    const int nx = J.cells[0], ny = J.cells[1], nz = J.cells[2], nc = nx * ny * nz;
    double *Te = work, *Tl = work + nc, *dE = work + 2 * nc;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        Te[c] = tp.T0;
        Tl[c] = tp.T0;
    }
    __syncthreads();
    const double delta = dt / J.substeps;
    double peak = tp.T0;
    for (int64_t n = 0; n < J.nsteps; ++n) {
        for (int k = 0; k < J.substeps; ++k) {
            const double tt = double(n) * dt + double(k) * delta;
            const double z = (tt - J.t0) / J.sigma_t;
            const double pulse = P0 * exp(-0.5 * z * z);
            for (int c = threadIdx.x; c < nc; c += blockDim.x) {
                const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
                const double Tc = Te[c];
                double lap = 0.0;
                if (nx > 1)
                    lap += (Te[(cz * ny + cy) * nx + (cx + 1) % nx] - 2.0 * Tc + Te[(cz * ny + cy) * nx + (cx + nx - 1) % nx]) /
                           (J.dx[0] * J.dx[0]);
                if (ny > 1)
                    lap += (Te[(cz * ny + (cy + 1) % ny) * nx + cx] - 2.0 * Tc + Te[(cz * ny + (cy + ny - 1) % ny) * nx + cx]) /
                           (J.dx[1] * J.dx[1]);
                if (nz > 1)
                    lap += (Te[(((cz + 1) % nz) * ny + cy) * nx + cx] - 2.0 * Tc +
                            Te[(((cz + nz - 1) % nz) * ny + cy) * nx + cx]) / (J.dx[2] * J.dx[2]);
                const double x = tp.G * (Tc - Tl[c]);
                dE[c] = delta * (tp.kappa_e * lap - x + pulse * J.shape[c]);
                Tl[c] += delta * x / tp.C_l;
            }
            __syncthreads();
            for (int c = threadIdx.x; c < nc; c += blockDim.x)
                Te[c] = sqrt(2.0 * (0.5 * tp.gamma_e * Te[c] * Te[c] + dE[c]) / tp.gamma_e);
            __syncthreads();
        }
        for (int c = threadIdx.x; c < nc; c += blockDim.x) peak = fmax(peak, Te[c]);
    }
    red[threadIdx.x] = peak;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// one CTA per (job, candidate power): the peak of a TTM-only run
__global__ void calibrate_kernel(const CalibJob *jobs, const double *cand, double *peaks, int ncand, double dt,
                                 TtmParams tp, int64_t work_per_block)
{
    __shared__ double red[1024];
    const int job = blockIdx.x / ncand;
    const CalibJob J = jobs[job];
    const double pk = calib_peak(J, cand[blockIdx.x], dt, tp, J.work + work_per_block * (blockIdx.x % ncand), red);
    if (threadIdx.x == 0) peaks[blockIdx.x] = pk;
}

}  // namespace

cudaError_t launch_calibrate(const CalibJob *jobs_dev, const double *cand_dev, double *peaks_dev, int njobs,
                             int ncand, int ncells, double dt, const TtmParams &tp, cudaStream_t st)
{
    if (njobs <= 0) return cudaSuccess;
    const int bs = ncells <= 32 ? 32 : (ncells <= 256 ? 256 : 1024);
    calibrate_kernel<<<njobs * ncand, bs, 0, st>>>(jobs_dev, cand_dev, peaks_dev, ncand, dt, tp, 3 * int64_t(ncells));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block size of the per-cell FP64 kernels (sigma table, TTM).  Their work is
// FP64 divisions, square roots and exponentials at about two FP64 FMAs a clock
// a SM, so a few thousand cells in 256-thread blocks would occupy a tenth of
// the SMs: take the largest power of two in [32, 256] that still gives a
// block to each of the 148 SMs.  Each thread computes the same cell either way.
// SMs of the current device (cached per device; 148 when it cannot be read).
static int device_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 148;
    }
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 148;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

// Threads a block for n independent work items: the largest of bs, bs/2, ...
// (down to one warp) that still gives every SM a block, so that a small
// launch spreads over the GPU instead of filling a few SMs (FP64 work runs
// at the FP64 rate of the SMs it lands on).
static int spread_block(int64_t n, int bs)
{
    const int sms = device_sms();
    while (bs > 32 && (n + bs - 1) / bs < sms) bs >>= 1;
    return bs;
}

static int cell_block(int64_t n) { return spread_block(n, 256); }

cudaError_t launch_sigma(const StepParams &p, const DevBuffers &b, int ncells, int precision, cudaStream_t st)
{
    // both tables: whichever one a pass reads holds the noise of the current T_e
    const int bs = cell_block(ncells), gs = (ncells + bs - 1) / bs;
    for (void *tab : {b.sigma, b.sigma_alt}) {
        if (!tab) continue;
        if (precision == 64)
            sigma_kernel<double><<<gs, bs, 0, st>>>(p, b.Te, static_cast<double *>(tab), ncells);
        else
            sigma_kernel<float><<<gs, bs, 0, st>>>(p, b.Te, static_cast<float *>(tab), ncells);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pass_general(const StepParams &p, const DevBuffers &b, int precision, int pass,
                                int64_t range_offset, int nranges, int64_t nwork, cudaStream_t st, int block,
                                SweepCtl sw)
{
    if (nwork <= 0) return cudaSuccess;
    const int bs = spread_block(nwork, block);
    const int64_t gs = (nwork + bs - 1) / bs;
    if (precision == 64)
        pass_general_kernel<double><<<gs, bs, 0, st>>>(p, b, pass, b.ranges + range_offset, nranges, nwork, sw);
    else
        pass_general_kernel<float><<<gs, bs, 0, st>>>(p, b, pass, b.ranges + range_offset, nranges, nwork, sw);
    return cudaGetLastError();
}

namespace {
__global__ void set_target_kernel(const int64_t *step, int64_t *target, int64_t n) { *target = *step + n; }
}  // namespace

cudaError_t launch_set_target(const DevBuffers &b, int64_t n, cudaStream_t st)
{
    set_target_kernel<<<1, 1, 0, st>>>(b.step, b.target, n);
    return cudaGetLastError();
}

cudaError_t launch_ttm(const StepParams &p, const DevBuffers &b, const TtmParams &tp, int n_instances,
                       cudaStream_t st, int precision, int inc_step)
{
    const int n = p.ncells_total, bs = cell_block(n), gs = (n + bs - 1) / bs;
    if (b.cell_inst && tp.source == TTS_SOURCE_STEP_PROFILE) {
        if (precision == 64)
            ttm_profile_kernel<double><<<gs, bs, 0, st>>>(p, b, tp, b.cell_inst, n);
        else
            ttm_profile_kernel<float><<<gs, bs, 0, st>>>(p, b, tp, b.cell_inst, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || !inc_step) return e;
        return launch_step_inc(b, st);
    }
    if (b.cell_inst && p.ttm_one_substep) {
        ttm_increment_kernel<<<gs, bs, 0, st>>>(p, b, tp, b.cell_inst, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (precision == 64)
            ttm_apply_kernel<double><<<gs, bs, 0, st>>>(p, b, tp, n, inc_step);
        else
            ttm_apply_kernel<float><<<gs, bs, 0, st>>>(p, b, tp, n, inc_step);
        return cudaGetLastError();
    }
    ttm_kernel<<<n_instances, 256, 0, st>>>(p, b, tp);
    return cudaGetLastError();
}

cudaError_t launch_obs(StepParams p, const DevBuffers &b, int precision, int nblocks, int mode, cudaStream_t st)
{
    const int grid = nblocks < 1184 ? nblocks : 1184;    // 8 CTAs per SM on 148 SMs
    p.obs_blocks = nblocks;
    if (precision == 64)
        obs_partial_kernel<double><<<grid, kObsBlock, 0, st>>>(p, b, mode);
    else
        obs_partial_kernel<float><<<grid, kObsBlock, 0, st>>>(p, b, mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_obs_reduce(p, b, mode, st);
}

cudaError_t launch_obs_reduce(const StepParams &p, const DevBuffers &b, int mode, cudaStream_t st)
{
    obs_reduce_kernel<<<p.n_instances, kObsReduceThreads, 0, st>>>(p, b, mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || mode != 0 || p.lattice_on) return e;
    step_inc_kernel<<<1, 1, 0, st>>>(b.step);
    return cudaGetLastError();
}

namespace {
// instance of a slot: the last instance whose first slot is <= slot
__device__ __forceinline__ int slot_instance(const DevInstance *inst, int n_inst, int64_t slot)
{
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].slot_begin <= slot) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename R>
__global__ void spins_to_atoms_kernel(const R *__restrict__ sx, const R *__restrict__ sy, const R *__restrict__ sz,
                                      const int *__restrict__ atom, const DevInstance *inst, int n_inst,
                                      int64_t n_total, R *out)
{
    const int64_t slot = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (slot >= n_total) return;
    const int64_t g = inst[slot_instance(inst, n_inst, slot)].slot_begin + atom[slot];
    out[3 * g] = sx[slot];
    out[3 * g + 1] = sy[slot];
    out[3 * g + 2] = sz[slot];
}

template <typename R>
__global__ void spins_from_atoms_kernel(R *sx, R *sy, R *sz, const int *__restrict__ atom, const DevInstance *inst,
                                        int n_inst, int64_t n_total, const R *__restrict__ in)
{
    const int64_t slot = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (slot >= n_total) return;
    const int64_t g = inst[slot_instance(inst, n_inst, slot)].slot_begin + atom[slot];
    sx[slot] = in[3 * g];
    sy[slot] = in[3 * g + 1];
    sz[slot] = in[3 * g + 2];
}
}  // namespace

cudaError_t launch_spins_to_atoms(const DevBuffers &b, int64_t n_total, int n_inst, int precision, void *out,
                                  cudaStream_t st)
{
    const int bs = 256;
    const int64_t gs = (n_total + bs - 1) / bs;
    if (precision == 64)
        spins_to_atoms_kernel<double><<<gs, bs, 0, st>>>(static_cast<const double *>(b.sx),
                                                         static_cast<const double *>(b.sy),
                                                         static_cast<const double *>(b.sz), b.atom, b.inst, n_inst,
                                                         n_total, static_cast<double *>(out));
    else
        spins_to_atoms_kernel<float><<<gs, bs, 0, st>>>(static_cast<const float *>(b.sx),
                                                        static_cast<const float *>(b.sy),
                                                        static_cast<const float *>(b.sz), b.atom, b.inst, n_inst,
                                                        n_total, static_cast<float *>(out));
    return cudaGetLastError();
}

cudaError_t launch_spins_from_atoms(const DevBuffers &b, int64_t n_total, int n_inst, int precision, const void *in,
                                    cudaStream_t st)
{
    const int bs = 256;
    const int64_t gs = (n_total + bs - 1) / bs;
    if (precision == 64)
        spins_from_atoms_kernel<double><<<gs, bs, 0, st>>>(static_cast<double *>(b.sx), static_cast<double *>(b.sy),
                                                           static_cast<double *>(b.sz), b.atom, b.inst, n_inst,
                                                           n_total, static_cast<const double *>(in));
    else
        spins_from_atoms_kernel<float><<<gs, bs, 0, st>>>(static_cast<float *>(b.sx), static_cast<float *>(b.sy),
                                                          static_cast<float *>(b.sz), b.atom, b.inst, n_inst, n_total,
                                                          static_cast<const float *>(in));
    return cudaGetLastError();
}

cudaError_t launch_step_inc(const DevBuffers &b, cudaStream_t st)
{
    step_inc_kernel<<<1, 1, 0, st>>>(b.step);
    return cudaGetLastError();
}

}  // namespace tts
