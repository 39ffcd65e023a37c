// tts_lattice.cu -- moving lattice (paper Sec. II.A): atoms under a
// shifted-force Morse potential plus the exchange-mediated force
// -dJ(r_ij)/dr (s_i.s_j), advanced together with the spins by
//   v += F dtL/2M; m/2 spin steps; x += v dtL; J(r_ij) refreshed;
//   m/2 spin steps; F recomputed; v += F dtL/2M;
//   exact Ornstein-Uhlenbeck electron-ion coupling with the kinetic-energy
//   change returned to the electrons of the atom's TTM cell; TTM by dtL.
//
// Layout: every atom keeps its reference lattice site (FP64) and its
// displacement u from it (spin precision), so pair vectors are the fixed
// reference vector of a candidate pair plus u_j - u_i.  Candidate pairs are
// all pairs within max(cutoffs) + skin of the reference lattice, in
// ascending atom id; an atom further than skin/2 from its site sets the
// health word.  The per-cell ion->electron energy is summed in 64-bit fixed
// point (2^-100 J), so the sum does not depend on the order of the atomics.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "tts_philox.cuh"
#include "tts_system.h"

namespace tts {

struct LatticeState {
    tts_lattice_desc d{};
    int m = 10;                 // spin steps per lattice step
    double dtL = 0.0, mass = 0.0;
    int zc = 0;                 // candidate width
    int64_t n = 0;
    double rc_J = 0.0;          // largest exchange cutoff
    int *cand = nullptr;        // [k][slot] candidate slot, -1 = none
    void *cvec = nullptr;       // [c][k][slot] reference pair vector (angstrom), spin precision
    double *ref = nullptr;      // [c][slot] reference position, angstrom
    void *u = nullptr;          // [c][slot] displacement, angstrom
    void *v = nullptr;          // [c][slot] velocity, m/s
    void *f = nullptr;          // [c][slot] force, N
    uint8_t *colour = nullptr;  // per slot
    int *inst_of = nullptr;     // per slot
    double *box = nullptr;      // [inst][3] angstrom
    long long *cell_acc = nullptr;   // per TTM cell, ion -> electron energy, units of 2^-100 J
    int64_t *lstep = nullptr;
    double *lat_partial = nullptr;   // per observable block: kinetic, pair energy
    int ncells_alloc = 0;
};

namespace {

constexpr double kFixScale = 1267650600228229401496703205376.0;   // 2^100

struct ExchTable {
    int kind[TTS_MAX_SPECIES][TTS_MAX_SPECIES];
    double J1[TTS_MAX_SPECIES][TTS_MAX_SPECIES], J2[TTS_MAX_SPECIES][TTS_MAX_SPECIES];
    double J3[TTS_MAX_SPECIES][TTS_MAX_SPECIES], rc[TTS_MAX_SPECIES][TTS_MAX_SPECIES];
};

struct LatArgs {
    int64_t n;
    int zc, zmax;
    const int *cand;
    const void *cvec;
    const double *ref;
    void *u, *v, *f;
    const uint8_t *colour;
    const int *inst_of;
    const double *box;
    long long *cell_acc;
    int64_t *lstep;
    double *lat_partial;
    ExchTable ex;
    double inv_mu[TTS_MAX_SPECIES];
    double morse_D, morse_alpha, morse_r0, morse_rc, dU_rc, U_rc;
    double mass, dtL, gamma_p, half_skin2;
    uint32_t key0, key1;
    int instance_base;
    int m;
    int sample_every;
};

template <typename R>
__device__ __forceinline__ R cv(const LatArgs &a, int c, int k, int64_t i)
{
    return static_cast<const R *>(a.cvec)[(int64_t(c) * a.zc + k) * a.n + i];
}

template <typename R>
__device__ __forceinline__ R *arr(void *p, int c, int64_t n)
{
    return static_cast<R *>(p) + int64_t(c) * n;
}

__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

// Bethe-Slater J(r) and its derivative, and the Morse force magnitude, in the
// spin precision R (FP32 systems compute their pair forces and exchange table
// in FP32; the force sums stay FP64).
template <typename R>
__device__ __forceinline__ R bethe_slater_dr_r(R r, R J1, R J2, R J3)
{
    const R x = (r / J3) * (r / J3);
    return R(4) * J1 * exp(-x) * (R(1) - R(2) * J2 * x - x + J2 * x * x) * R(2) * r / (J3 * J3);
}

template <typename R>
__device__ __forceinline__ R bethe_slater_r(R r, R J1, R J2, R J3)
{
    const R x = (r / J3) * (r / J3);
    return R(4) * J1 * x * (R(1) - J2 * x) * exp(-x);
}

template <typename R>
__device__ __forceinline__ R morse_dU_raw_r(const LatArgs &a, R r)
{
    const R e1 = exp(-R(a.morse_alpha) * (r - R(a.morse_r0)));
    return R(2) * R(a.morse_alpha) * R(a.morse_D) * (e1 - e1 * e1);
}

__device__ __forceinline__ double morse_U_raw(const LatArgs &a, double r)
{
    const double e1 = exp(-a.morse_alpha * (r - a.morse_r0));
    return a.morse_D * (e1 * e1 - 2.0 * e1);
}

template <typename R>
__global__ void kick_kernel(LatArgs a, double coef)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    for (int c = 0; c < 3; ++c) {
        R *v = arr<R>(a.v, c, a.n);
        const R *f = arr<R>(a.f, c, a.n);
        v[i] = static_cast<R>(double(v[i]) + double(f[i]) * coef);
    }
}

template <typename R>
__global__ void drift_kernel(LatArgs a, unsigned int *health)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        R *u = arr<R>(a.u, c, a.n);
        const R *v = arr<R>(a.v, c, a.n);
        const double x = double(u[i]) + double(v[i]) * a.dtL * 1e10;
        u[i] = static_cast<R>(x);
        d2 += x * x;
    }
    if (d2 > a.half_skin2) atomicOr(health, kHealthSkin);
}

// exchange table J(r)/mu_i for the current positions (ascending candidate =
// ascending atom id), colour check, bath cell of every atom
template <typename R>
__global__ void refresh_kernel(LatArgs a, DevBuffers b, int precision_is_64)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const R *ux = arr<R>(a.u, 0, a.n), *uy = arr<R>(a.u, 1, a.n), *uz = arr<R>(a.u, 2, a.n);
    const int ti = b.species[i];
    int cnt = 0;
    R *w = static_cast<R *>(b.nbr_w);
    for (int k = 0; k < a.zc; ++k) {
        const int j = a.cand[int64_t(k) * a.n + i];
        if (j < 0) break;
        const int tj = b.species[j];
        const int kind = a.ex.kind[ti][tj];
        if (kind == TTS_EXCH_NONE) continue;
        const R dx = cv<R>(a, 0, k, i) + (ux[j] - ux[i]);
        const R dy = cv<R>(a, 1, k, i) + (uy[j] - uy[i]);
        const R dz = cv<R>(a, 2, k, i) + (uz[j] - uz[i]);
        const R r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r < R(a.ex.rc[ti][tj]))) continue;
        // J(r) / mu_i in the spin precision (tesla), J1 / mu_i folded first
        const R J = kind == TTS_EXCH_CONST
                        ? R(a.ex.J1[ti][tj] * a.inv_mu[ti])
                        : bethe_slater_r<R>(r, R(a.ex.J1[ti][tj] * a.inv_mu[ti]), R(a.ex.J2[ti][tj]), R(a.ex.J3[ti][tj]));
        if (J == R(0)) continue;
        if (a.colour[i] == a.colour[j]) atomicOr(b.health, kHealthColour);
        if (cnt >= a.zmax) {
            atomicOr(b.health, kHealthOverflow);
            break;
        }
        b.nbr[int64_t(cnt) * a.n + i] = j;
        w[int64_t(cnt) * a.n + i] = J;
        ++cnt;
    }
    for (; cnt < a.zmax; ++cnt) {
        b.nbr[int64_t(cnt) * a.n + i] = static_cast<int>(i);
        w[int64_t(cnt) * a.n + i] = R(0);
    }
    // TTM cell of the atom from its current position, floor(x / L * n)
    const int inst = a.inst_of[i];
    const DevInstance I = b.inst[inst];
    int cc[3];
    const R *uc[3] = {ux, uy, uz};
    for (int c = 0; c < 3; ++c) {
        const double L = a.box[3 * inst + c];
        double x = a.ref[int64_t(c) * a.n + i] + double(uc[c][i]);
        x -= L * floor(x / L);
        if (x >= L) x -= L;
        const double fr = x / L;
        int q = static_cast<int>(floor(fr * I.cells[c]));
        cc[c] = q >= I.cells[c] ? I.cells[c] - 1 : (q < 0 ? 0 : q);
    }
    b.cell[i] = I.cell_begin + (cc[2] * I.cells[1] + cc[1]) * I.cells[0] + cc[0];
    (void)precision_is_64;
}

template <typename R>
__global__ void force_kernel(LatArgs a, DevBuffers b)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const R *ux = arr<R>(a.u, 0, a.n), *uy = arr<R>(a.u, 1, a.n), *uz = arr<R>(a.u, 2, a.n);
    const R *S0 = static_cast<const R *>(b.sx), *S1 = static_cast<const R *>(b.sy), *S2 = static_cast<const R *>(b.sz);
    const int ti = b.species[i];
    const R si0 = S0[i], si1 = S1[i], si2 = S2[i];
    const R uxi = ux[i], uyi = uy[i], uzi = uz[i];
    // pair terms in the spin precision, energies in units of 1e-20 J inside
    // the loop so that FP32 stays far from its range limits; the sums are
    // compensated (each addition's rounding error carried in a second word,
    // Knuth's TwoSum), which keeps their rounding near that of FP64 sums at
    // the spin precision's rate.  Products are rounded before they are
    // added (no fused multiply-add), as TwoSum assumes.
    const R morse_rc = R(a.morse_rc), dU_rc = R(a.dU_rc * 1e20);
    R fx = R(0), fy = R(0), fz = R(0), ex = R(0), ey = R(0), ez = R(0);
    auto two_sum = [](R &sum, R &err, R v) {
        const R t = sum + v;
        const R bp = t - sum;
        err += (sum - (t - bp)) + (v - bp);
        sum = t;
    };
    for (int k = 0; k < a.zc; ++k) {
        const int j = a.cand[int64_t(k) * a.n + i];
        if (j < 0) break;
        const R dx = cv<R>(a, 0, k, i) + (ux[j] - uxi);
        const R dy = cv<R>(a, 1, k, i) + (uy[j] - uyi);
        const R dz = cv<R>(a, 2, k, i) + (uz[j] - uzi);
        const R r = sqrt(dx * dx + dy * dy + dz * dz);
        R g = R(0);                                      // dE_pair/dr, 1e-20 J per angstrom
        if (r < morse_rc) g += morse_dU_raw_r<R>(a, r) * R(1e20) - dU_rc;
        const int tj = b.species[j];
        if (a.ex.kind[ti][tj] == TTS_EXCH_BETHE_SLATER && r < R(a.ex.rc[ti][tj])) {
            const R ss = si0 * S0[j] + si1 * S1[j] + si2 * S2[j];
            g -= bethe_slater_dr_r<R>(r, R(a.ex.J1[ti][tj] * 1e20), R(a.ex.J2[ti][tj]), R(a.ex.J3[ti][tj])) * ss;
        }
        if (g != R(0)) {
            const R s = g / r;                           // 1e-20 J per angstrom^2
            two_sum(fx, ex, mul_rn(s, dx));
            two_sum(fy, ey, mul_rn(s, dy));
            two_sum(fz, ez, mul_rn(s, dz));
        }
    }
    // 1e-20 J per angstrom = 1e-10 N
    arr<R>(a.f, 0, a.n)[i] = static_cast<R>((double(fx) + double(ex)) * 1e-10);
    arr<R>(a.f, 1, a.n)[i] = static_cast<R>((double(fy) + double(ey)) * 1e-10);
    arr<R>(a.f, 2, a.n)[i] = static_cast<R>((double(fz) + double(ez)) * 1e-10);
}

// second half kick, then the Ornstein-Uhlenbeck electron-ion coupling
template <typename R>
__global__ void kick_ou_kernel(LatArgs a, DevBuffers b, double coef)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double vv[3];
    for (int c = 0; c < 3; ++c) {
        R *v = arr<R>(a.v, c, a.n);
        vv[c] = static_cast<double>(static_cast<R>(double(v[i]) + double(arr<R>(a.f, c, a.n)[i]) * coef));
        v[i] = static_cast<R>(vv[c]);
    }
    if (!(a.gamma_p > 0.0)) return;
    const double c1 = exp(-a.gamma_p * a.dtL / a.mass);
    const int cell = b.cell[i];
    const double T = b.Te[cell];
    const double c2 = sqrt(kBoltzmann * T * (1.0 - c1 * c1) / a.mass);
    const u32x4 w = philox4x32_10(u32x4{static_cast<uint32_t>(b.atom[i]), static_cast<uint32_t>(*a.lstep), 0xFFFF0002u,
                                        static_cast<uint32_t>(a.instance_base + a.inst_of[i])},
                                  a.key0, a.key1);
    const double u0 = uniform_d(w.x), u1 = uniform_d(w.y), u2 = uniform_d(w.z), u3 = uniform_d(w.w);
    const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    double s1, co1, s3, co3;
    sincospi(2.0 * u1, &s1, &co1);
    sincospi(2.0 * u3, &s3, &co3);
    const double g[3] = {r01 * co1, r01 * s1, r23 * co3};
    double ke0 = 0.0, ke1 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double v1 = c1 * vv[c] + c2 * g[c];
        ke0 += 0.5 * a.mass * vv[c] * vv[c];
        ke1 += 0.5 * a.mass * v1 * v1;
        arr<R>(a.v, c, a.n)[i] = static_cast<R>(v1);
    }
    const long long q = llrint(-(ke1 - ke0) * kFixScale);
    atomicAdd(reinterpret_cast<unsigned long long *>(a.cell_acc + cell), static_cast<unsigned long long>(q));
}

// TTM of a moving lattice: ion energy handed over, then diffusion and the
// source over dtL in sub-steps (no G term: the ions couple through their own
// friction and noise).  One cluster of kLatTtmCtas CTAs per instance (16, the
// largest cluster the part allows with the non-portable size), each CTA
// a contiguous range of its cells: the grid's FP64 work spreads over that many
// SMs (one SM's FP64 rate made a single block take ~0.9 ms a lattice step on
// a 10 x 10 x 40 grid with 13 sub-steps).  T_e and the increments live in
// global memory; cluster barriers (release / acquire) order the phases.
constexpr int kLatTtmCtas = 16;
constexpr int kLatTtmThreads = 256;

__device__ __forceinline__ void lat_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__global__ void __launch_bounds__(kLatTtmThreads) lattice_ttm_kernel(LatArgs a, DevBuffers b, TtmParams tp)
{
    const int inst = static_cast<int>(blockIdx.x) / kLatTtmCtas, rank = static_cast<int>(blockIdx.x) % kLatTtmCtas;
    const DevInstance I = b.inst[inst];
    const int nc = I.ncells;
    const int c0 = static_cast<int>(int64_t(rank) * nc / kLatTtmCtas);
    const int c1 = static_cast<int>(int64_t(rank + 1) * nc / kLatTtmCtas);
    double *Te = b.Te + I.cell_begin;
    double *dE = b.ttm_scratch + I.cell_begin;
    const double *shape = b.src_shape + I.cell_begin;
    for (int c = c0 + static_cast<int>(threadIdx.x); c < c1; c += blockDim.x) {
        const long long q = a.cell_acc[I.cell_begin + c];
        a.cell_acc[I.cell_begin + c] = 0;
        if (q != 0) {
            const double Ee = 0.5 * tp.gamma_e * Te[c] * Te[c] + (double(q) / kFixScale) / I.cell_volume;
            Te[c] = sqrt(2.0 * Ee * tp.inv_gamma_e);
        }
    }
    lat_cluster_sync();
    const int64_t ls = *a.lstep;
    const double delta = a.dtL / I.substeps;
    double deposited = 0.0;
    const int nxc = I.cells[0], nyc = I.cells[1], nzc = I.cells[2];
    for (int k = 0; k < I.substeps; ++k) {
        const double t = double(ls) * a.dtL + double(k) * delta;
        double pulse = 0.0;
        if (tp.source != TTS_SOURCE_NONE) {
            const double z = (t - I.t0) / I.sigma_t;
            pulse = I.P0 * exp(-0.5 * z * z);
        }
        for (int c = c0 + static_cast<int>(threadIdx.x); c < c1; c += blockDim.x) {
            const int cx = c % nxc, cy = (c / nxc) % nyc, cz = c / (nxc * nyc);
            const double Tc = Te[c];
            double lap = 0.0;
            if (nxc > 1)
                lap += (Te[(cz * nyc + cy) * nxc + (cx + 1) % nxc] - 2.0 * Tc + Te[(cz * nyc + cy) * nxc + (cx + nxc - 1) % nxc]) *
                       I.inv_dx2[0];
            if (nyc > 1)
                lap += (Te[(cz * nyc + (cy + 1) % nyc) * nxc + cx] - 2.0 * Tc + Te[(cz * nyc + (cy + nyc - 1) % nyc) * nxc + cx]) *
                       I.inv_dx2[1];
            if (nzc > 1)
                lap += (Te[(((cz + 1) % nzc) * nyc + cy) * nxc + cx] - 2.0 * Tc +
                        Te[(((cz + nzc - 1) % nzc) * nyc + cy) * nxc + cx]) * I.inv_dx2[2];
            const double src = pulse * shape[c];
            dE[c] = delta * (tp.kappa_e * lap + src);
            deposited += delta * src * I.cell_volume;
        }
        lat_cluster_sync();
        for (int c = c0 + static_cast<int>(threadIdx.x); c < c1; c += blockDim.x)
            Te[c] = sqrt(2.0 * (0.5 * tp.gamma_e * Te[c] * Te[c] + dE[c]) * tp.inv_gamma_e);
        lat_cluster_sync();
    }
    // source energy deposited: threads in a fixed tree, then the CTAs in rank
    // order by CTA 0 through distributed shared memory
    __shared__ double red[kLatTtmThreads];
    red[threadIdx.x] = deposited;
    __syncthreads();
    for (int h = kLatTtmThreads / 2; h > 0; h >>= 1) {
        if (static_cast<int>(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    lat_cluster_sync();
    if (rank == 0 && threadIdx.x == 0) {
        double tot = 0.0;
        const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(&red[0]));
        for (int r = 0; r < kLatTtmCtas; ++r) {
            uint32_t remote;
            double v;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
            asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
            tot += v;
        }
        b.src_energy[inst] += tot;
    }
    lat_cluster_sync();        // no CTA leaves while CTA 0 may still read its partial
}

// kinetic and pair energies per observable block (sampling steps only)
template <typename R>
__global__ void __launch_bounds__(kObsBlock) lattice_energy_kernel(LatArgs a, DevBuffers b)
{
    if (a.sample_every <= 0 || (*a.lstep + 1) % a.sample_every != 0) return;
    const int inst = b.obs_block_inst[blockIdx.x];
    const DevInstance I = b.inst[inst];
    double e[2] = {0.0, 0.0};    // kinetic, pair
    const R *ux = arr<R>(a.u, 0, a.n), *uy = arr<R>(a.u, 1, a.n), *uz = arr<R>(a.u, 2, a.n);
    for (int jj = 0; jj < kObsSpan / kObsBlock; ++jj) {
        const int64_t i = b.obs_block_begin[blockIdx.x] + threadIdx.x + int64_t(jj) * kObsBlock;
        if (i >= I.slot_begin + I.n) break;
        for (int c = 0; c < 3; ++c) {
            const double v = arr<R>(a.v, c, a.n)[i];
            e[0] += 0.5 * a.mass * v * v;
        }
        for (int k = 0; k < a.zc; ++k) {
            const int j = a.cand[int64_t(k) * a.n + i];
            if (j < 0) break;
            const double dx = double(cv<R>(a, 0, k, i)) + double(ux[j]) - double(ux[i]);
            const double dy = double(cv<R>(a, 1, k, i)) + double(uy[j]) - double(uy[i]);
            const double dz = double(cv<R>(a, 2, k, i)) + double(uz[j]) - double(uz[i]);
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < a.morse_rc) e[1] += 0.5 * (morse_U_raw(a, r) - a.U_rc - (r - a.morse_rc) * a.dU_rc);
        }
    }
    block_sum_store<2>(e, a.lat_partial + 2 * int64_t(blockIdx.x));
}

__global__ void inc_kernel(int64_t *counter) { *counter += 1; }

// host-side candidate pairs of one lattice instance: every site within rcut of
// the atom's site (minimum image), ascending atom id, with the reference vector
void lattice_candidates(const tts_system_desc &d, const HostInstance &hi, double rcut,
                        std::vector<std::vector<std::pair<int64_t, std::array<double, 3>>>> *out)
{
    static const int basis[3][4][3] = {{{0, 0, 0}}, {{0, 0, 0}, {1, 1, 1}}, {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}}};
    static const int nbasis[3] = {1, 2, 4};
    const int lat = d.lattice, nb = nbasis[lat];
    const int reach = static_cast<int>(std::ceil(rcut / d.a)) + 1;
    const int *L = hi.cells;
    out->assign(hi.n, {});
    for (int64_t i = 0; i < hi.n; ++i) {
        const int b = static_cast<int>(i % nb);
        const int64_t cell = i / nb;
        const int ix = static_cast<int>(cell % L[0]), iy = static_cast<int>((cell / L[0]) % L[1]);
        const int iz = static_cast<int>(cell / (int64_t(L[0]) * L[1]));
        auto &row = (*out)[i];
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dx = -reach; dx <= reach; ++dx)
                    for (int b2 = 0; b2 < nb; ++b2) {
                        const int hx = 2 * dx + basis[lat][b2][0] - basis[lat][b][0];
                        const int hy = 2 * dy + basis[lat][b2][1] - basis[lat][b][1];
                        const int hz = 2 * dz + basis[lat][b2][2] - basis[lat][b][2];
                        const double r = 0.5 * d.a * std::sqrt(double(hx * hx + hy * hy + hz * hz));
                        if (!(r > 0.0 && r < rcut)) continue;
                        const int jx = ((ix + dx) % L[0] + L[0]) % L[0];
                        const int jy = ((iy + dy) % L[1] + L[1]) % L[1];
                        const int jz = ((iz + dz) % L[2] + L[2]) % L[2];
                        const int64_t j = ((int64_t(jz) * L[1] + jy) * L[0] + jx) * nb + b2;
                        row.push_back({j, {0.5 * d.a * hx, 0.5 * d.a * hy, 0.5 * d.a * hz}});
                    }
        std::sort(row.begin(), row.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    }
}

LatArgs make_args(tts_system *s)
{
    LatticeState *L = s->lat;
    LatArgs a{};
    a.n = L->n;
    a.zc = L->zc;
    a.zmax = s->zmax;
    a.cand = L->cand;
    a.cvec = L->cvec;
    a.ref = L->ref;
    a.u = L->u;
    a.v = L->v;
    a.f = L->f;
    a.colour = L->colour;
    a.inst_of = L->inst_of;
    a.box = L->box;
    a.cell_acc = L->cell_acc;
    a.lstep = L->lstep;
    a.lat_partial = L->lat_partial;
    for (int x = 0; x < TTS_MAX_SPECIES; ++x) {
        a.inv_mu[x] = s->p.sp[x].mu > 0.0 ? 1.0 / s->p.sp[x].mu : 0.0;
        for (int y = 0; y < TTS_MAX_SPECIES; ++y) {
            const tts_exchange &e = s->desc.exch[x][y];
            a.ex.kind[x][y] = (x < s->desc.nspecies && y < s->desc.nspecies) ? e.kind : TTS_EXCH_NONE;
            a.ex.J1[x][y] = e.J1;
            a.ex.J2[x][y] = e.J2;
            a.ex.J3[x][y] = e.J3;
            a.ex.rc[x][y] = e.rc;
        }
    }
    const tts_lattice_desc &d = L->d;
    a.morse_D = d.morse_D;
    a.morse_alpha = d.morse_alpha;
    a.morse_r0 = d.morse_r0;
    a.morse_rc = d.morse_rc;
    {
        const double e1 = std::exp(-d.morse_alpha * (d.morse_rc - d.morse_r0));
        a.U_rc = d.morse_D * (e1 * e1 - 2.0 * e1);
        a.dU_rc = 2.0 * d.morse_alpha * d.morse_D * (e1 - e1 * e1);
    }
    a.mass = L->mass;
    a.dtL = L->dtL;
    a.gamma_p = d.gamma_p;
    a.half_skin2 = 0.25 * d.skin * d.skin;
    a.key0 = s->p.key0;
    a.key1 = s->p.key1;
    a.instance_base = s->desc.instance_base;
    a.m = L->m;
    a.sample_every = s->desc.sample_every;
    return a;
}

template <typename R>
cudaError_t launch_per_atom(tts_system *s, cudaStream_t st, int which, double coef)
{
    const LatArgs a = make_args(s);
    const int bs = 256;
    const int64_t gs = (a.n + bs - 1) / bs;
    switch (which) {
    case 0: kick_kernel<R><<<gs, bs, 0, st>>>(a, coef); break;
    case 1: drift_kernel<R><<<gs, bs, 0, st>>>(a, s->b.health); break;
    case 2: refresh_kernel<R><<<gs, bs, 0, st>>>(a, s->b, s->precision == 64); break;
    case 3: force_kernel<R><<<gs, bs, 0, st>>>(a, s->b); break;
    case 4: kick_ou_kernel<R><<<gs, bs, 0, st>>>(a, s->b, coef); break;
    case 5: lattice_energy_kernel<R><<<s->obs_blocks, kObsBlock, 0, st>>>(a, s->b); break;
    default: break;
    }
    return cudaGetLastError();
}

cudaError_t per_atom(tts_system *s, cudaStream_t st, int which, double coef = 0.0)
{
    return s->precision == 64 ? launch_per_atom<double>(s, st, which, coef) : launch_per_atom<float>(s, st, which, coef);
}

}  // namespace

void lattice_destroy(LatticeState *L)
{
    if (!L) return;
    for (void *q : {static_cast<void *>(L->cand), L->cvec, static_cast<void *>(L->ref), L->u, L->v, L->f,
                    static_cast<void *>(L->colour), static_cast<void *>(L->inst_of), static_cast<void *>(L->box),
                    static_cast<void *>(L->cell_acc), static_cast<void *>(L->lstep), static_cast<void *>(L->lat_partial)})
        if (q) cudaFree(q);
    delete L;
}

int64_t lattice_units_per_step(const tts_system *s) { return s->lat ? s->n_total * s->lat->m : s->n_total; }

double lattice_step_length(const tts_system *s) { return s->lat ? s->lat->dtL : s->desc.dt; }

// Checkpoint part of a moving lattice: lattice step, u, v, f (3 x n each,
// spin precision), per-cell tallies.  With buf == nullptr only the size.
size_t lattice_state_bytes(const tts_system *s)
{
    if (!s->lat) return 0;
    return sizeof(int64_t) + 9 * size_t(s->n_total) * s->rsize + size_t(s->lat->ncells_alloc) * sizeof(long long);
}

int lattice_state_io(tts_system *s, char *buf, bool save)
{
    LatticeState *L = s->lat;
    if (!L) return TTS_OK;
    const cudaMemcpyKind k = save ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    auto io = [&](void *dev, size_t bytes) -> cudaError_t {
        cudaError_t e = save ? cudaMemcpy(buf, dev, bytes, k) : cudaMemcpy(dev, buf, bytes, k);
        buf += bytes;
        return e;
    };
    const size_t arr = 3 * size_t(s->n_total) * s->rsize;
    cudaError_t e = io(L->lstep, sizeof(int64_t));
    if (e == cudaSuccess) e = io(L->u, arr);
    if (e == cudaSuccess) e = io(L->v, arr);
    if (e == cudaSuccess) e = io(L->f, arr);
    if (e == cudaSuccess && L->ncells_alloc > 0) e = io(L->cell_acc, size_t(L->ncells_alloc) * sizeof(long long));
    if (e != cudaSuccess) return cuda_fail(e, "lattice state");
    // the exchange table and bath cells follow the restored positions
    return save ? TTS_OK : lattice_refresh_tables(s);
}

int lattice_refresh_tables(tts_system *s)
{
    cudaError_t e = per_atom(s, s->stream, 2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    ++s->launches;
    return e == cudaSuccess ? TTS_OK : cuda_fail(e, "lattice refresh");
}

// recompute the exchange table, cells and forces for the current state
int lattice_refresh_now(tts_system *s)
{
    cudaError_t e = per_atom(s, s->stream, 2);
    if (e == cudaSuccess) e = per_atom(s, s->stream, 3);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    s->launches += 2;
    return e == cudaSuccess ? TTS_OK : cuda_fail(e, "lattice refresh");
}

int lattice_ensure_cell_acc(tts_system *s)
{
    LatticeState *L = s->lat;
    if (L->ncells_alloc >= s->ncells_total) return TTS_OK;
    if (L->cell_acc) cudaFree(L->cell_acc);
    L->cell_acc = nullptr;
    int rc = dev_alloc(&L->cell_acc, s->ncells_total, "ion energy tallies");
    if (rc) return rc;
    TTS_CUDA(cudaMemsetAsync(L->cell_acc, 0, s->ncells_total * sizeof(long long), s->stream), "zero tallies");
    L->ncells_alloc = s->ncells_total;
    return TTS_OK;
}

cudaError_t lattice_record_step(tts_system *s, cudaStream_t st, int *kernels, cudaEvent_t ev0, cudaEvent_t ev1)
{
    LatticeState *L = s->lat;
    *kernels = 0;
    cudaError_t e = cudaSuccess;
    if (ev0) e = cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal);
    const double coef = L->dtL / (2.0 * L->mass);
    if (e == cudaSuccess) { e = launch_sigma(s->p, s->b, s->ncells_total, s->precision, st); ++*kernels; }
    if (e == cudaSuccess) { e = per_atom(s, st, 0, coef); ++*kernels; }
    for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
        for (int k = 0; k < L->m / 2 && e == cudaSuccess; ++k) {
            for (int pass = 0; pass < s->max_passes && e == cudaSuccess; ++pass) {
                const int64_t off = s->pass_offset[pass];
                const int nr = static_cast<int>(s->pass_offset[pass + 1] - off);
                e = launch_pass_general(s->p, s->b, s->precision, pass, off, nr, s->pass_work[pass], st, s->pass_block);
                ++*kernels;
            }
            if (e == cudaSuccess) {
                inc_kernel<<<1, 1, 0, st>>>(s->b.step);
                e = cudaGetLastError();
                ++*kernels;
            }
        }
        if (half == 0 && e == cudaSuccess) {
            e = per_atom(s, st, 1);
            if (e == cudaSuccess) e = per_atom(s, st, 2);
            *kernels += 2;
        }
    }
    if (e == cudaSuccess) { e = per_atom(s, st, 3); ++*kernels; }
    if (e == cudaSuccess) { e = per_atom(s, st, 4, coef); ++*kernels; }
    if (e == cudaSuccess && s->ttm_active) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(s->n_inst * kLatTtmCtas));
        cfg.blockDim = dim3(kLatTtmThreads);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kLatTtmCtas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaFuncSetAttribute(lattice_ttm_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, lattice_ttm_kernel, make_args(s), s->b, s->tp);
        if (e == cudaSuccess) e = cudaGetLastError();
        ++*kernels;
    }
    if (e == cudaSuccess && s->desc.sample_every > 0) {
        e = per_atom(s, st, 5);
        ++*kernels;
        if (e == cudaSuccess) {
            StepParams p = s->p;
            p.lattice_on = 1;
            p.lstep = L->lstep;
            p.lat_partial = L->lat_partial;
            e = launch_obs(p, s->b, s->precision, s->obs_blocks, 0, st);
            *kernels += 2;
        }
    }
    if (e == cudaSuccess) {
        inc_kernel<<<1, 1, 0, st>>>(L->lstep);
        e = cudaGetLastError();
        ++*kernels;
    }
    if (e == cudaSuccess && ev1) e = cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    return e;
}

}  // namespace tts

using namespace tts;

extern "C" {

int tts_set_lattice(tts_system *s, const tts_lattice_desc *d)
{
    if (!s || !d) return fail(TTS_ERR_ARG, "null argument");
    if (s->lat) return fail(TTS_ERR_STATE, "the lattice already moves");
    if (s->ttm_active) return fail(TTS_ERR_STATE, "switch the moving lattice on before setting the TTM grid");
    if (s->desc.lattice == TTS_LATTICE_CLUSTER) return fail(TTS_ERR_UNSUPPORTED, "clusters have no lattice to move");
    if (s->eng) return fail(TTS_ERR_UNSUPPORTED, "a moving lattice runs on the general engine (engine = general)");
    if (s->merged) return fail(TTS_ERR_UNSUPPORTED, "the merged sweep is for rigid lattices");
    if (d->spin_substeps < 2 || d->spin_substeps % 2) return fail(TTS_ERR_ARG, "spin_substeps must be even and >= 2");
    if (!(d->mass_amu > 0.0) || !(d->morse_rc > 0.0) || !(d->morse_alpha > 0.0) || !(d->skin >= 0.0) ||
        !(d->T_init >= 0.0) || !(d->gamma_p >= 0.0))
        return fail(TTS_ERR_ARG, "lattice parameters out of range");
    double rc_J = 0.0;
    for (int x = 0; x < s->desc.nspecies; ++x)
        for (int y = 0; y < s->desc.nspecies; ++y)
            if (s->desc.exch[x][y].kind != TTS_EXCH_NONE) rc_J = std::max(rc_J, s->desc.exch[x][y].rc);
    const double rcut = std::max(rc_J, d->morse_rc) + d->skin;
    for (const HostInstance &hi : s->host)
        for (int k = 0; k < 3; ++k)
            if (!(hi.box[k] > 2.0 * rcut)) return fail(TTS_ERR_ARG, "box edges must exceed twice (cutoff + skin)");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set lattice");
    LatticeState *L = new LatticeState;
    L->d = *d;
    L->m = d->spin_substeps;
    L->dtL = d->spin_substeps * s->desc.dt;
    L->mass = d->mass_amu * 1.66053906660e-27;
    L->n = s->n_total;
    L->rc_J = rc_J;
    const int64_t N = s->n_total;
    const size_t rs = s->rsize;
    // candidates
    std::vector<std::vector<std::vector<std::pair<int64_t, std::array<double, 3>>>>> cands(s->n_inst);
    int zc = 0;
    for (int i = 0; i < s->n_inst; ++i) {
        lattice_candidates(s->desc, s->host[i], rcut, &cands[i]);
        for (auto &row : cands[i]) zc = std::max<int>(zc, static_cast<int>(row.size()));
    }
    L->zc = zc;
    std::vector<int> cand(size_t(zc) * N, -1), inst_of(N);
    std::vector<double> cvec_d(3 * size_t(zc) * N, 0.0), ref(3 * N), u(3 * N, 0.0), v(3 * N, 0.0), box(3 * s->n_inst);
    std::vector<uint8_t> colour(N);
    for (int i = 0; i < s->n_inst; ++i) {
        const HostInstance &hi = s->host[i];
        const DevInstance &di = s->dinst[i];
        for (int k = 0; k < 3; ++k) box[3 * i + k] = hi.box[k];
        const double Lz = hi.box[2];
        // initial velocities: Maxwell-Boltzmann from Philox, net momentum removed
        std::vector<double> vel(3 * hi.n);
        double mean[3] = {0.0, 0.0, 0.0};
        const double vs = std::sqrt(kBoltzmann * d->T_init / L->mass);
        for (int64_t a = 0; a < hi.n; ++a) {
            const u32x4 w = philox4x32_10(u32x4{static_cast<uint32_t>(a), 0u, 0xFFFF0003u,
                                                static_cast<uint32_t>(s->desc.instance_base + i)},
                                          s->p.key0, s->p.key1);
            const double u0 = uniform_d(w.x), u1 = uniform_d(w.y), u2 = uniform_d(w.z), u3 = uniform_d(w.w);
            const double r01 = std::sqrt(-2.0 * std::log(u0)), r23 = std::sqrt(-2.0 * std::log(u2));
            const double g[3] = {r01 * std::cos(2.0 * M_PI * u1), r01 * std::sin(2.0 * M_PI * u1),
                                 r23 * std::cos(2.0 * M_PI * u3)};
            for (int k = 0; k < 3; ++k) {
                vel[3 * a + k] = vs * g[k];
                mean[k] += vel[3 * a + k];
            }
        }
        for (int64_t a = 0; a < hi.n; ++a) {
            const int64_t slot = di.slot_begin + s->slot_of_atom[i][a];
            inst_of[slot] = i;
            colour[slot] = static_cast<uint8_t>(hi.colour[a]);
            for (int k = 0; k < 3; ++k) {
                ref[k * N + slot] = hi.pos[3 * a + k];
                v[k * N + slot] = vel[3 * a + k] - mean[k] / hi.n;
            }
            // initial longitudinal strain wave along z, one wavelength per box
            const double z0 = hi.pos[3 * a + 2];
            u[2 * N + slot] = d->strain_amp * Lz / (2.0 * M_PI) * std::sin(2.0 * M_PI * z0 / Lz);
            const auto &row = cands[i][a];
            for (size_t k = 0; k < row.size(); ++k) {
                cand[k * N + slot] = static_cast<int>(di.slot_begin + s->slot_of_atom[i][row[k].first]);
                for (int c = 0; c < 3; ++c) cvec_d[(size_t(c) * zc + k) * N + slot] = row[k].second[c];
            }
        }
    }
    // exchange table width: the rigid count plus a margin (overflow sets the health word)
    int rc = TTS_OK;
    char *q = nullptr;
    auto alloc_r = [&](void **p, size_t count, const char *what) {
        if (rc) return;
        rc = dev_alloc(&q, count * rs, what);
        *p = q;
    };
    if (!rc) rc = dev_alloc(&L->cand, cand.size(), "candidate pairs");
    alloc_r(&L->cvec, cvec_d.size(), "candidate vectors");
    if (!rc) rc = dev_alloc(&L->ref, ref.size(), "reference sites");
    alloc_r(&L->u, 3 * N, "displacements");
    alloc_r(&L->v, 3 * N, "velocities");
    alloc_r(&L->f, 3 * N, "forces");
    if (!rc) rc = dev_alloc(&L->colour, N, "colours");
    if (!rc) rc = dev_alloc(&L->inst_of, N, "instance of atom");
    if (!rc) rc = dev_alloc(&L->box, box.size(), "boxes");
    if (!rc) rc = dev_alloc(&L->lstep, 1, "lattice step");
    if (!rc) rc = dev_alloc(&L->lat_partial, 2 * size_t(s->obs_blocks), "lattice partials");
    if (rc) {
        lattice_destroy(L);
        return rc;
    }
    auto up_r = [&](void *dst, const std::vector<double> &src, const char *what) {
        if (rc) return;
        if (s->precision == 64) {
            rc = upload(dst, src.data(), src.size() * sizeof(double), s->stream, what);
        } else {
            std::vector<float> tmp(src.begin(), src.end());
            rc = upload(dst, tmp.data(), tmp.size() * sizeof(float), s->stream, what);
        }
    };
    rc = upload(L->cand, cand.data(), cand.size() * sizeof(int), s->stream, "upload candidates");
    up_r(L->cvec, cvec_d, "upload candidate vectors");
    if (!rc) rc = upload(L->ref, ref.data(), ref.size() * sizeof(double), s->stream, "upload sites");
    up_r(L->u, u, "upload displacements");
    up_r(L->v, v, "upload velocities");
    if (!rc) rc = upload(L->colour, colour.data(), colour.size(), s->stream, "upload colours");
    if (!rc) rc = upload(L->inst_of, inst_of.data(), inst_of.size() * sizeof(int), s->stream, "upload instances");
    if (!rc) rc = upload(L->box, box.data(), box.size() * sizeof(double), s->stream, "upload boxes");
    if (rc) {
        lattice_destroy(L);
        return rc;
    }
    TTS_CUDA(cudaMemsetAsync(L->lstep, 0, sizeof(int64_t), s->stream), "zero lattice step");
    s->lat = L;
    if ((rc = lattice_ensure_cell_acc(s))) return rc;
    s->dirty = true;
    return lattice_refresh_now(s);
}

int tts_get_positions(tts_system *s, int inst, double *xyz)
{
    if (!s || !xyz || inst < 0 || inst >= s->n_inst) return fail(TTS_ERR_ARG, "bad argument");
    const HostInstance &hi = s->host[inst];
    const DevInstance &di = s->dinst[inst];
    const int64_t N = s->n_total;
    std::vector<double> u(3 * di.n, 0.0);
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get positions");
    if (s->lat) {
        for (int c = 0; c < 3; ++c) {
            if (s->precision == 64) {
                TTS_CUDA(cudaMemcpy(u.data() + c * di.n, static_cast<double *>(s->lat->u) + c * N + di.slot_begin,
                                    di.n * sizeof(double), cudaMemcpyDeviceToHost), "read displacements");
            } else {
                std::vector<float> tmp(di.n);
                TTS_CUDA(cudaMemcpy(tmp.data(), static_cast<float *>(s->lat->u) + c * N + di.slot_begin,
                                    di.n * sizeof(float), cudaMemcpyDeviceToHost), "read displacements");
                for (int64_t k = 0; k < di.n; ++k) u[c * di.n + k] = tmp[k];
            }
        }
    }
    for (int64_t a = 0; a < hi.n; ++a) {
        const int64_t sl = s->slot_of_atom[inst][a];
        for (int c = 0; c < 3; ++c) {
            double x = hi.pos[3 * a + c] + u[c * di.n + sl];
            if (hi.box[c] > 0.0) {
                x -= hi.box[c] * std::floor(x / hi.box[c]);
                if (x >= hi.box[c]) x -= hi.box[c];
            }
            xyz[3 * a + c] = x;
        }
    }
    return TTS_OK;
}

int tts_get_velocities(tts_system *s, int inst, double *xyz)
{
    if (!s || !xyz || inst < 0 || inst >= s->n_inst) return fail(TTS_ERR_ARG, "bad argument");
    if (!s->lat) return fail(TTS_ERR_STATE, "the lattice does not move");
    const DevInstance &di = s->dinst[inst];
    const int64_t N = s->n_total;
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get velocities");
    std::vector<double> v(3 * di.n);
    for (int c = 0; c < 3; ++c) {
        if (s->precision == 64) {
            TTS_CUDA(cudaMemcpy(v.data() + c * di.n, static_cast<double *>(s->lat->v) + c * N + di.slot_begin,
                                di.n * sizeof(double), cudaMemcpyDeviceToHost), "read velocities");
        } else {
            std::vector<float> tmp(di.n);
            TTS_CUDA(cudaMemcpy(tmp.data(), static_cast<float *>(s->lat->v) + c * N + di.slot_begin,
                                di.n * sizeof(float), cudaMemcpyDeviceToHost), "read velocities");
            for (int64_t k = 0; k < di.n; ++k) v[c * di.n + k] = tmp[k];
        }
    }
    for (int64_t a = 0; a < di.n; ++a) {
        const int64_t sl = s->slot_of_atom[inst][a];
        for (int c = 0; c < 3; ++c) xyz[3 * a + c] = v[c * di.n + sl];
    }
    return TTS_OK;
}

}  // extern "C"
