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
template <typename R>
__global__ void sigma_kernel(StepParams p, const double *__restrict__ Te, R *__restrict__ sigma, int ncells)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncells) return;
    const double T = Te[g];
    for (int t = 0; t < TTS_MAX_SPECIES; ++t)
        for (int hs = 0; hs < 2; ++hs) {
            double v = 0.0;
            if (t < p.nspecies && T > 0.0 && p.sp[t].alpha > 0.0) {
                const double h = hs ? p.dt : 0.5 * p.dt;
                v = sqrt(2.0 * p.sp[t].alpha * kBoltzmann * T / (kGyro * p.sp[t].mu * h));
            }
            sigma[(g * TTS_MAX_SPECIES + t) * 2 + hs] = static_cast<R>(v);
        }
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
__global__ void __launch_bounds__(256) pass_general_kernel(StepParams p, DevBuffers b, int pass,
                                                           const PassRange *__restrict__ ranges, int nranges,
                                                           int64_t nwork)
{
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
    const R h = r.hsel ? R(p.dt) : R(0.5 * p.dt);
    const R sig = static_cast<const R *>(b.sigma)[(int64_t(b.cell[slot]) * TTS_MAX_SPECIES + t) * 2 + r.hsel];
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
// Observables.  mode 0: inside a step (sample when (step+1) % every == 0, into
// the ring, then advance the step counter); mode 1: now, into obs_now.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kObsBlock) obs_partial_kernel(StepParams p, DevBuffers b, int mode)
{
    const int64_t step = *b.step;
    const int64_t clock = p.lattice_on ? *p.lstep : step;
    if (mode == 0 && (p.sample_every <= 0 || (clock + 1) % p.sample_every != 0)) return;
    const int inst = b.obs_block_inst[blockIdx.x];
    const DevInstance I = b.inst[inst];
    const int64_t first = b.obs_block_begin[blockIdx.x];
    const int64_t end = I.slot_begin + I.n;
    double acc[kObsFields];
#pragma unroll
    for (int k = 0; k < kObsFields; ++k) acc[k] = 0.0;
    const R *S0 = static_cast<const R *>(b.sx), *S1 = static_cast<const R *>(b.sy), *S2 = static_cast<const R *>(b.sz);
    const int64_t slot = first + threadIdx.x;
    if (slot < end) {
        const int t = b.species[slot];
        const double sx = S0[slot], sy = S1[slot], sz = S2[slot];
        // exchange part alone (for the pair energy), then the full field
        double hx = 0, hy = 0, hz = 0;
        const R *w = static_cast<const R *>(b.nbr_w);
        for (int k = 0; k < p.zmax; ++k) {
            const int64_t e = int64_t(k) * p.n_total + slot;
            const double J = w[e];
            const int j = b.nbr[e];
            hx += J * double(S0[j]);
            hy += J * double(S1[j]);
            hz += J * double(S2[j]);
        }
        const double mu = p.sp[t].mu;
        const double sn = sx * p.axis[0] + sy * p.axis[1] + sz * p.axis[2];
        const double ka = p.sp[t].kappa * sn;
        const double Bx = hx + ka * p.axis[0] + p.B[0];
        const double By = hy + ka * p.axis[1] + p.B[1];
        const double Bz = hz + ka * p.axis[2] + p.B[2];
        const double Hx = mu * Bx, Hy = mu * By, Hz = mu * Bz;
        const double cx = sy * Hz - sz * Hy, cy = sz * Hx - sx * Hz, cz = sx * Hy - sy * Hx;
        double *a = acc + 12 * t;
        a[0] = 1.0;
        a[1] = sx; a[2] = sy; a[3] = sz;
        a[7] = -0.5 * mu * (sx * hx + sy * hy + sz * hz);
        a[8] = -p.sp[t].K * sn * sn;
        a[9] = -mu * (p.B[0] * sx + p.B[1] * sy + p.B[2] * sz);
        a[10] = cx * cx + cy * cy + cz * cz;
        a[11] = sx * Hx + sy * Hy + sz * Hz;
    }
    __shared__ double red[kObsBlock];
    for (int k = 0; k < kObsFields; ++k) {
        red[threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = kObsBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) b.obs_partial[int64_t(blockIdx.x) * kObsFields + k] = red[0];
        __syncthreads();
    }
}

// Per species t the partial sums are, at 12 t + k: k = 0 count, 1..3 sum s,
// 4..6 unused, 7 exchange energy (half of mu s.h per atom, each pair counted
// twice), 8 anisotropy, 9 Zeeman, 10 sum |s x H|^2, 11 sum s.H.  The moment-
// weighted direction is sum_t mu_t sum_{i in t} s_i / sum_t mu_t n_t.
__global__ void obs_final_kernel(StepParams p, DevBuffers b, int mode)
{
    const int64_t step = *b.step;
    const int64_t clock = p.lattice_on ? *p.lstep : step;
    const bool sample = (mode == 1) || (p.sample_every > 0 && (clock + 1) % p.sample_every == 0);
    if (sample) {
        for (int inst = threadIdx.x; inst < p.n_instances; inst += blockDim.x) {
            const DevInstance I = b.inst[inst];
            double tot[kObsFields];
            for (int k = 0; k < kObsFields; ++k) tot[k] = 0.0;
            for (int blk = I.obs_block_begin; blk < I.obs_block_begin + I.obs_block_count; ++blk)
                for (int k = 0; k < kObsFields; ++k) tot[k] += b.obs_partial[int64_t(blk) * kObsFields + k];
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
            double te = 0.0, tl = 0.0;
            for (int c = 0; c < I.ncells; ++c) {
                te += b.Te[I.cell_begin + c];
                tl += b.Tl[I.cell_begin + c];
            }
            rec[15] = te / I.ncells;
            rec[16] = tl / I.ncells;
            if (p.lattice_on && mode == 0) {
                double ek = 0.0, em = 0.0;
                for (int blk = I.obs_block_begin; blk < I.obs_block_begin + I.obs_block_count; ++blk) {
                    ek += p.lat_partial[2 * int64_t(blk)];
                    em += p.lat_partial[2 * int64_t(blk) + 1];
                }
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
    }
    __syncthreads();
    if (mode == 0 && !p.lattice_on && threadIdx.x == 0) *b.step = step + 1;
}

// ---------------------------------------------------------------------------
// Source calibration, one block per job.  The TTM-only run uses the same
// update as ttm_kernel; every thread keeps the running maximum of its cells
// and the block reduces it once per run.
// ---------------------------------------------------------------------------
__device__ double calib_peak(CalibJob &J, double P0, double dt, const TtmParams &tp, double *red)
{
    const int nx = J.cells[0], ny = J.cells[1], nz = J.cells[2], nc = nx * ny * nz;
    double *Te = J.work, *Tl = J.work + nc, *dE = J.work + 2 * nc;
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

__global__ void calibrate_kernel(CalibJob *jobs, double dt, TtmParams tp)
{
    __shared__ double red[256];
    CalibJob &J = jobs[blockIdx.x];
    double hi = J.guess;
    // at most 200 doublings: the peak grows without bound with P0
    for (int it = 0; it < 200 && calib_peak(J, hi, dt, tp, red) < J.target; ++it) hi *= 2.0;
    double lo = 0.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (calib_peak(J, mid, dt, tp, red) < J.target) lo = mid; else hi = mid;
    }
    if (threadIdx.x == 0) J.P0 = 0.5 * (lo + hi);
}

}  // namespace

cudaError_t launch_calibrate(CalibJob *jobs_dev, int njobs, int ncells, double dt, const TtmParams &tp, cudaStream_t st)
{
    if (njobs <= 0) return cudaSuccess;
    calibrate_kernel<<<njobs, ncells <= 32 ? 32 : 256, 0, st>>>(jobs_dev, dt, tp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
cudaError_t launch_sigma(const StepParams &p, const DevBuffers &b, int ncells, int precision, cudaStream_t st)
{
    const int bs = 128, gs = (ncells + bs - 1) / bs;
    if (precision == 64)
        sigma_kernel<double><<<gs, bs, 0, st>>>(p, b.Te, static_cast<double *>(b.sigma), ncells);
    else
        sigma_kernel<float><<<gs, bs, 0, st>>>(p, b.Te, static_cast<float *>(b.sigma), ncells);
    return cudaGetLastError();
}

cudaError_t launch_pass_general(const StepParams &p, const DevBuffers &b, int precision, int pass,
                                int64_t range_offset, int nranges, int64_t nwork, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    const int bs = 256;
    const int64_t gs = (nwork + bs - 1) / bs;
    if (precision == 64)
        pass_general_kernel<double><<<gs, bs, 0, st>>>(p, b, pass, b.ranges + range_offset, nranges, nwork);
    else
        pass_general_kernel<float><<<gs, bs, 0, st>>>(p, b, pass, b.ranges + range_offset, nranges, nwork);
    return cudaGetLastError();
}

cudaError_t launch_ttm(const StepParams &p, const DevBuffers &b, const TtmParams &tp, int n_instances,
                       cudaStream_t st)
{
    ttm_kernel<<<n_instances, 256, 0, st>>>(p, b, tp);
    return cudaGetLastError();
}

cudaError_t launch_obs(const StepParams &p, const DevBuffers &b, int precision, int nblocks, int mode,
                       cudaStream_t st)
{
    if (precision == 64)
        obs_partial_kernel<double><<<nblocks, kObsBlock, 0, st>>>(p, b, mode);
    else
        obs_partial_kernel<float><<<nblocks, kObsBlock, 0, st>>>(p, b, mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    obs_final_kernel<<<1, 256, 0, st>>>(p, b, mode);
    return cudaGetLastError();
}

}  // namespace tts
