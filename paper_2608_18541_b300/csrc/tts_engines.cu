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
#include "tts_bulk.cuh"
#include "tts_pair.cuh"
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
    typename Vec4<R>::T *S;      // all instances, general slot order
    const int *cell;             // general slot -> TTM cell
    const R *sigma;              // [cell][species][h]
    const int64_t *step;
    unsigned int *health;
    FastSpecies<R> sp[TTS_MAX_SPECIES];
    R nx, ny, nz, Bx, By, Bz;
    R dt;
    uint32_t key0, key1;
    uint32_t Lx, Ly, Lz, hx;     // shape shared by all instances
    uint32_t nkx;                // blocks along the hx colour sites of a row
    FastDiv dnkx;                // division by nkx (by 1 where nkx = 0)
    uint32_t nhalf;              // sites per colour
    int64_t n_inst_sites;        // sites per instance
    uint32_t inst_base;          // global id of instance 0
    SweepCtl sw;                 // merged sweep: leading / trailing colour-0 pass
};

// One colour pass, one site per thread.  Block (BX, BY) threads cover BX
// consecutive colour sites of BY rows; grid (ceil(hx / BX) * ceil(Ly / BY),
// Lz, instances).  All instances share one shape, so no per-thread index needs
// a division.
// At most 256 threads a block; in FP32 six blocks per SM (40 registers a
// thread), so that 48 warps hide the neighbour-load latency.
template <typename R, bool AXZ>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1) checker_pass_kernel(CheckerArgs<R> a, int colour, int hsel, int pass)
{
    using V = typename Vec4<R>::T;
    {
        int hd = -1;
        if (a.sw.mode != 0 && !sweep_gate(a.sw, a.step, hd)) return;
        if (hd >= 0) hsel = hd;
    }
    // block index -> (row block, x block); the quotient is uniform over the block
    const uint32_t yb = blockIdx.x / a.nkx;
    const uint32_t kx = (blockIdx.x - yb * a.nkx) * blockDim.x + threadIdx.x;
    const uint32_t y = yb * blockDim.y + threadIdx.y;
    const uint32_t hx = a.hx, Ly = a.Ly, Lz = a.Lz;
    if (y >= Ly || kx >= hx) return;
    const uint32_t z = blockIdx.y;
    const int inst = blockIdx.z;
    V *S = a.S + int64_t(inst) * a.n_inst_sites;
    const V *O = S + (colour ? 0 : a.nhalf);
    V *Own = S + (colour ? a.nhalf : 0);
    const uint32_t zp = (z + 1 == Lz) ? 0 : z + 1, zm = (z == 0) ? Lz - 1 : z - 1;
    const uint32_t yp = (y + 1 == Ly) ? 0 : y + 1, ym = (y == 0) ? Ly - 1 : y - 1;
    const uint32_t row = z * Ly + y;
    const uint32_t par = (y + z + colour) & 1u;
    const uint32_t x = 2 * kx + par;
    // x neighbours: the other colour's sites kx and kx +- 1 (periodic in hx)
    uint32_t kxp, kxm;
    if (par) {
        kxp = (kx + 1 == hx) ? 0 : kx + 1;
        kxm = kx;
    } else {
        kxp = kx;
        kxm = (kx == 0) ? hx - 1 : kx - 1;
    }
    const uint32_t k = row * hx + kx;
    const V n0 = O[(zp * Ly + y) * hx + kx];
    const V n1 = O[(zm * Ly + y) * hx + kx];
    const V n2 = O[(z * Ly + yp) * hx + kx];
    const V n3 = O[(z * Ly + ym) * hx + kx];
    const V n4 = O[row * hx + kxp];
    const V n5 = O[row * hx + kxm];
    V own = Own[k];
    const R htx = n0.x + n1.x + n2.x + n3.x + n4.x + n5.x;
    const R hty = n0.y + n1.y + n2.y + n3.y + n4.y + n5.y;
    const R htz = n0.z + n1.z + n2.z + n3.z + n4.z + n5.z;
    const R h1x = n0.w * n0.x + n1.w * n1.x + n2.w * n2.x + n3.w * n3.x + n4.w * n4.x + n5.w * n5.x;
    const R h1y = n0.w * n0.y + n1.w * n1.y + n2.w * n2.y + n3.w * n3.y + n4.w * n4.y + n5.w * n5.y;
    const R h1z = n0.w * n0.z + n1.w * n1.z + n2.w * n2.z + n3.w * n3.z + n4.w * n4.z + n5.w * n5.z;
    const int t = own.w != R(0) ? 1 : 0;
    const FastSpecies<R> sp = t ? a.sp[1] : a.sp[0];
    const int *cell = a.cell + int64_t(inst) * a.n_inst_sites + (colour ? a.nhalf : 0);
    const R sig = a.sigma[(cell[k] * TTS_MAX_SPECIES + t) * 2 + hsel];
    const R h = hsel ? a.dt : R(0.5) * a.dt;
    R sx = own.x, sy = own.y, sz = own.z;
    if (sig > R(0)) {
        const uint32_t atom = row * a.Lx + x;
        const u32x4 w = philox4x32_10(
            u32x4{atom, static_cast<uint32_t>(*a.step), static_cast<uint32_t>(pass), a.inst_base + inst}, a.key0,
            a.key1);
        fast_update<R, AXZ>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, sp, a.nx, a.ny, a.nz, a.Bx, a.By, a.Bz, sig, &w,
                            h);
    } else {
        fast_update<R, AXZ>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, sp, a.nx, a.ny, a.nz, a.Bx, a.By, a.Bz, sig,
                            nullptr, h);
    }
    // a non-finite component makes the sum non-finite
    if (!isfinite(sx + sy + sz)) atomicOr(a.health, kHealthNonFinite);
    own.x = sx;
    own.y = sy;
    own.z = sz;
    Own[k] = own;
}

// ---------------------------------------------------------------------------
// FP32 checkerboard engine on site pairs.  Rows y and y + Ly/2 of one colour
// are paired lane-wise: per instance and colour, pair q = (z Ly/2 + y) hx + kx
// (y < Ly/2) is stored as two 16-byte words in two planes,
//   lo plane: (x_A, x_B, y_A, y_B)      hi plane: (z_A, z_B, w_A, w_B),
// A = row y, B = row y + Ly/2, w = species flag.  The neighbours of a pair in
// z and x are pairs in the same lane order, in y too except across the row
// Ly/2 - 1 | 0 boundary, where lanes swap.  Every load is a ready f32x2
// operand, so the whole update runs on the packed FP32 pipe.
// ---------------------------------------------------------------------------
struct PairArgs {
    ulonglong2 *S;               // all instances: [inst][colour][lo | hi plane][pair]
    ulonglong2 *S1;              // second state buffer of the fused sweep (= S without it)
    const int *cur;              // 1: the current state is in S1, else in S
    const int *cell;             // general slot -> TTM cell
    const float *sigma;          // [cell][species][h], the table of this launch's step
    const int64_t *step;
    unsigned int *health;
    PairConsts k;
    PhiloxRoundKeys rk;
    uint32_t Lx, Ly, Lz, hx, Ly2;
    uint32_t nkx;                // blocks along the hx colour sites of a row
    FastDiv dnkx;                // division by nkx (by 1 where nkx = 0)
    uint32_t nhalf;              // sites per colour
    uint32_t npair;              // pairs per colour (nhalf / 2)
    int64_t n_inst_sites;
    uint32_t inst_base;
    int noise;                   // some species has alpha > 0 (else sigma = 0 everywhere)
    int n_inst;
    int inst0;                   // first instance of the launch (grid z counts from it)
    // TTM cell of a site from its coordinates, cell0 + inst cstride +
    // (cz ncy + cy) ncx + cx with c_k = floor(k n_k / L_k); the host checks it
    // against the cell map, else cell_formula = 0 and the map is read.
    int cell_formula;
    int cell0, cstride;
    uint32_t ncx, ncy, ncz;
    FastDiv dLx, dLy, dLz;
    int shx, shy, shz;           // >= 0: L_k / n_k = 2^sh, c_k = k >> sh
    SweepCtl sw;                 // merged sweep: leading / trailing colour-0 pass
    int pf_planes;               // L2 prefetch distance in z planes (0: none)
};

struct Pair4 {
    f2 x, y, z, w;
};

// The buffer holding the current state: the fused sweep reads one buffer and
// writes the other, then flips *cur; every other kernel of the pair layout
// works on the current buffer in place.
__device__ __forceinline__ ulonglong2 *pair_state(const PairArgs &a) { return *a.cur ? a.S1 : a.S; }

__device__ __forceinline__ Pair4 load_pair(const ulonglong2 *lo, const ulonglong2 *hi, uint32_t q)
{
    const ulonglong2 a = lo[q], b = hi[q];
    return Pair4{f2{a.x}, f2{a.y}, f2{b.x}, f2{b.y}};
}

__device__ __forceinline__ Pair4 swap_lanes(const Pair4 &n)
{
    return Pair4{f2_swap(n.x), f2_swap(n.y), f2_swap(n.z), f2_swap(n.w)};
}

__device__ __forceinline__ void add_neighbour(const Pair4 &n, f2 &htx, f2 &hty, f2 &htz, f2 &h1x, f2 &h1y, f2 &h1z)
{
    htx = htx + n.x;
    hty = hty + n.y;
    htz = htz + n.z;
    h1x = fma2(n.w, n.x, h1x);
    h1y = fma2(n.w, n.y, h1y);
    h1z = fma2(n.w, n.z, h1z);
}

// Where a pair sits: instance, plane z, pair row y2 < Ly/2, colour site kx,
// and the x parities of its two rows.
struct PairSite {
    int inst;
    uint32_t z, y2, kx, parA, parB;
};

__device__ __forceinline__ PairSite make_site(const PairArgs &a, int inst, uint32_t z, uint32_t y2, uint32_t kx,
                                              int colour)
{
    PairSite p;
    p.inst = inst;
    p.z = z;
    p.y2 = y2;
    p.kx = kx;
    p.parA = (y2 + z + uint32_t(colour)) & 1u;
    p.parB = p.parA ^ (a.Ly2 & 1u);
    return p;
}

// Thermal directions of the pair (Philox counters: atom, step, pass, global
// instance); independent of any loaded value.
__device__ __forceinline__ void site_noise(const PairArgs &a, const PairSite &p, uint32_t step, int pass, f2 &g1,
                                           f2 &g2, f2 &g3)
{
    const uint32_t ig = a.inst_base + uint32_t(p.inst);
    const uint32_t atomA = (p.z * a.Ly + p.y2) * a.Lx + 2 * p.kx + p.parA;
    const uint32_t atomB = (p.z * a.Ly + p.y2 + a.Ly2) * a.Lx + 2 * p.kx + p.parB;
    pair_noise(u32x4{atomA, step, static_cast<uint32_t>(pass), ig}, u32x4{atomB, step, static_cast<uint32_t>(pass), ig},
               a.rk, a.k, g1, g2, g3);
}

// Neighbour sums of a pair from one z plane's tile of the other colour (rows
// ry-1, ry, ry+1 of the tile hold pair rows y2-1, y2, y2+1) and the two
// planes z +- 1 (row ry).  Sum order: z+1, z-1, y+1, y-1, x, x'.
__device__ __forceinline__ void neighbour_sums(const PairSite &p, uint32_t hx, uint32_t Ly2, const ulonglong2 *Pz_lo,
                                               const ulonglong2 *Pz_hi, const ulonglong2 *Pp_lo,
                                               const ulonglong2 *Pp_hi, const ulonglong2 *Pm_lo,
                                               const ulonglong2 *Pm_hi, uint32_t rp, uint32_t rm,
                                               uint32_t r0, uint32_t ryp, uint32_t rym, f2 &htx, f2 &hty, f2 &htz,
                                               f2 &h1x, f2 &h1y, f2 &h1z)
{
    const uint32_t kx = p.kx;
    const uint32_t kxp = (kx + 1 == hx) ? 0 : kx + 1, kxm = (kx == 0) ? hx - 1 : kx - 1;
    htx = hty = htz = h1x = h1y = h1z = f2{0};
    add_neighbour(load_pair(Pp_lo, Pp_hi, rp + kx), htx, hty, htz, h1x, h1y, h1z);
    add_neighbour(load_pair(Pm_lo, Pm_hi, rm + kx), htx, hty, htz, h1x, h1y, h1z);
    {
        Pair4 n = load_pair(Pz_lo, Pz_hi, ryp + kx);
        if (p.y2 + 1 == Ly2) n = swap_lanes(n);     // pair row 0 with lanes swapped
        add_neighbour(n, htx, hty, htz, h1x, h1y, h1z);
    }
    {
        Pair4 n = load_pair(Pz_lo, Pz_hi, rym + kx);
        if (p.y2 == 0) n = swap_lanes(n);           // pair row Ly/2 - 1 with lanes swapped
        add_neighbour(n, htx, hty, htz, h1x, h1y, h1z);
    }
    // x neighbours: the other colour's sites kx and kx + 1 (odd x) or kx - 1
    // (even x); with Ly/2 odd the two lanes differ in parity
    add_neighbour(load_pair(Pz_lo, Pz_hi, r0 + kx), htx, hty, htz, h1x, h1y, h1z);
    if (p.parA == p.parB) {
        add_neighbour(load_pair(Pz_lo, Pz_hi, r0 + (p.parA ? kxp : kxm)), htx, hty, htz, h1x, h1y, h1z);
    } else {
        const Pair4 P = load_pair(Pz_lo, Pz_hi, r0 + kxp), M = load_pair(Pz_lo, Pz_hi, r0 + kxm);
        const Pair4 &LA = p.parA ? P : M, &LB = p.parA ? M : P;
        add_neighbour(Pair4{f2_mix(LA.x, LB.x), f2_mix(LA.y, LB.y), f2_mix(LA.z, LB.z), f2_mix(LA.w, LB.w)}, htx,
                      hty, htz, h1x, h1y, h1z);
    }
}

// How a pair kernel finds the TTM cell of a site: from the cell map, from the
// coordinates by shifts (every L_k / n_k a power of two) or by invariant
// division, fixed at launch; or chosen per site at run time.
enum PairCellMode { kCellMap = 0, kCellShift = 1, kCellDiv = 2, kCellAny = 3 };

// TTM cells of the two sites of a pair.
template <int CM>
__device__ __forceinline__ void pair_cells(const PairArgs &a, const PairSite &p, int colour, int &cA, int &cB)
{
    if (CM == kCellMap || (CM == kCellAny && !a.cell_formula)) {
        // general slots of the two sites within the instance
        const uint32_t slotA = uint32_t(colour) * a.nhalf + (p.z * a.Ly + p.y2) * a.hx + p.kx;
        const uint32_t slotB = slotA + a.Ly2 * a.hx;
        const int *cell = a.cell + int64_t(p.inst) * a.n_inst_sites;
        cA = cell[slotA];
        cB = cell[slotB];
        return;
    }
    // c_k = floor(k n_k / L_k)
    auto cc = [&](uint32_t v, uint32_t n, const FastDiv &d, int sh) {
        if (CM == kCellShift) return v >> sh;
        if (CM == kCellDiv) return fast_div(v * n, d);
        return sh >= 0 ? v >> sh : fast_div(v * n, d);
    };
    const uint32_t cz = cc(p.z, a.ncz, a.dLz, a.shz);
    const uint32_t cyA = cc(p.y2, a.ncy, a.dLy, a.shy), cyB = cc(p.y2 + a.Ly2, a.ncy, a.dLy, a.shy);
    const uint32_t cxA = cc(2 * p.kx + p.parA, a.ncx, a.dLx, a.shx);
    const uint32_t cxB = cc(2 * p.kx + p.parB, a.ncx, a.dLx, a.shx);
    const int base = a.cell0 + p.inst * a.cstride;
    cA = base + int((cz * a.ncy + cyA) * a.ncx + cxA);
    cB = base + int((cz * a.ncy + cyB) * a.ncx + cxB);
}

// Update the pair from its neighbour sums and own words and store it at pair
// q of the own colour's planes.
template <bool AXZ, int CM = kCellAny>
__device__ __forceinline__ void pair_finish(const PairArgs &a, const PairSite &p, int colour, int hsel, bool h2, f2 g1,
                                            f2 g2, f2 g3, f2 htx, f2 hty, f2 htz, f2 h1x, f2 h1y, f2 h1z,
                                            ulonglong2 olo, ulonglong2 ohi, ulonglong2 *Wlo, ulonglong2 *Whi,
                                            uint32_t q)
{
    f2 sx{olo.x}, sy{olo.y}, sz{ohi.x};
    const f2 w{ohi.y};
    f2 sig{0};
    if (a.noise) {
        float wA, wB;
        f2_split(w, wA, wB);
        const int tA = wA != 0.0f ? 1 : 0, tB = wB != 0.0f ? 1 : 0;
        int cA, cB;
        pair_cells<CM>(a, p, colour, cA, cB);
        sig = f2_make(a.sigma[(cA * TTS_MAX_SPECIES + tA) * 2 + hsel], a.sigma[(cB * TTS_MAX_SPECIES + tB) * 2 + hsel]);
    }
    pair_update<AXZ>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, w, a.noise != 0, sig, g1, g2, g3, a.k, h2);
    float sA, sB;
    f2_split(sx + sy + sz, sA, sB);
    // a non-finite component makes the sum non-finite
    if (!isfinite(sA) || !isfinite(sB)) atomicOr(a.health, kHealthNonFinite);
    Wlo[q] = ulonglong2{sx.v, sy.v};
    Whi[q] = ulonglong2{sz.v, ohi.y};
}

// One colour pass, one site pair per thread, neighbours read from global
// memory.  Block (BX, BY) covers BX consecutive pairs of BY pair rows; grid
// (ceil(hx / BX) * ceil(Ly/2 / BY), Lz, instances).  Registers are capped at
// 64 (four 256-thread blocks a SM); a budget of 85 with fewer threads in
// flight measured slower.
// One block's worth of pairs: block index bx of a row of blocks (BX pairs x
// BY pair rows), plane z, instance inst.
template <bool AXZ, int CM>
__device__ __forceinline__ void pair_block(const PairArgs &a, int colour, int hsel, bool h2, int pass, uint32_t bx,
                                           uint32_t z, int inst)
{
    const uint32_t yb = fast_div(bx, a.dnkx);
    const uint32_t kx = (bx - yb * a.nkx) * blockDim.x + threadIdx.x;
    const uint32_t y2 = yb * blockDim.y + threadIdx.y;
    const uint32_t hx = a.hx, Ly2 = a.Ly2, Lz = a.Lz;
    // One thread asks the copy engine to bring this block's rows of both
    // colours at plane z + pf_planes into L2 (bulk prefetch, no registers, no
    // completion to wait for): the blocks that will read them -- the same rows
    // a few planes on, and their z neighbours -- then hit L2 instead of HBM.
    if (a.pf_planes > 0 && threadIdx.x == 0 && threadIdx.y == 0 && z + a.pf_planes < Lz) {
        const uint32_t zf = z + a.pf_planes, y0 = yb * blockDim.y, kx0 = (bx - yb * a.nkx) * blockDim.x;
        const uint32_t rows = min(blockDim.y, Ly2 - y0), cols = min(blockDim.x, hx - kx0);
        const ulonglong2 *ib = pair_state(a) + int64_t(inst) * a.n_inst_sites;
        for (uint32_t r = 0; r < rows; ++r) {
            const uint32_t q = (zf * Ly2 + y0 + r) * hx + kx0;
            bulk_prefetch_l2(ib + q, cols * 16u);                           // colour 0, lo plane
            bulk_prefetch_l2(ib + a.npair + q, cols * 16u);                 // colour 0, hi plane
            bulk_prefetch_l2(ib + a.nhalf + q, cols * 16u);                 // colour 1, lo plane
            bulk_prefetch_l2(ib + a.nhalf + a.npair + q, cols * 16u);       // colour 1, hi plane
        }
    }
    if (y2 >= Ly2 || kx >= hx) return;
    const PairSite p = make_site(a, inst, z, y2, kx, colour);
    f2 g1{0}, g2{0}, g3{0};
    if (a.noise) site_noise(a, p, static_cast<uint32_t>(*a.step), pass, g1, g2, g3);
    ulonglong2 *base = pair_state(a) + int64_t(inst) * a.n_inst_sites;
    const ulonglong2 *Olo = base + (colour ? 0 : a.nhalf);
    const ulonglong2 *Ohi = Olo + a.npair;
    ulonglong2 *Wlo = base + (colour ? a.nhalf : 0);
    ulonglong2 *Whi = Wlo + a.npair;
    const uint32_t zp = (z + 1 == Lz) ? 0 : z + 1, zm = (z == 0) ? Lz - 1 : z - 1;
    const uint32_t yp = (y2 + 1 == Ly2) ? 0 : y2 + 1, ym = (y2 == 0) ? Ly2 - 1 : y2 - 1;
    const uint32_t r0 = (z * Ly2 + y2) * hx;
    f2 htx, hty, htz, h1x, h1y, h1z;
    neighbour_sums(p, hx, Ly2, Olo, Ohi, Olo, Ohi, Olo, Ohi, (zp * Ly2 + y2) * hx, (zm * Ly2 + y2) * hx, r0,
                   (z * Ly2 + yp) * hx, (z * Ly2 + ym) * hx, htx, hty, htz, h1x, h1y, h1z);
    const uint32_t q = r0 + kx;
    pair_finish<AXZ, CM>(a, p, colour, hsel, h2, g1, g2, g3, htx, hty, htz, h1x, h1y, h1z, Wlo[q], Whi[q], Wlo, Whi,
                         q);
}

// SW: the launch is a leading or trailing pass of the merged sweep (compiled
// apart so that the other passes carry none of its code).  Those run on a
// persistent grid that walks the (row block, z, instance) blocks, so that a
// trailing pass the sweep skips costs one early exit per resident CTA.
template <bool AXZ, bool SW, int CM>
__global__ void __launch_bounds__(256, 4) checker_pair_kernel(PairArgs a, int colour, int hsel, int pass)
{
    if (!SW) {
        pair_block<AXZ, CM>(a, colour, hsel, false, pass, blockIdx.x, blockIdx.y, a.inst0 + static_cast<int>(blockIdx.z));
        return;
    }
    int hd = -1;
    if (!sweep_gate(a.sw, a.step, hd)) return;
    const bool h2 = hd == 1;          // constants made for dt/2, the bridge runs dt
    if (hd >= 0) hsel = hd;
    const uint32_t nbx = a.nkx * ((a.Ly2 + blockDim.y - 1) / blockDim.y);
    const uint64_t nvb = uint64_t(nbx) * a.Lz * uint64_t(a.n_inst);
    for (uint64_t v = blockIdx.x; v < nvb; v += gridDim.x) {
        const uint32_t bx = static_cast<uint32_t>(v % nbx);
        const uint64_t r = v / nbx;
        pair_block<AXZ, CM>(a, colour, hsel, h2, pass, bx, static_cast<uint32_t>(r % a.Lz), static_cast<int>(r / a.Lz));
    }
}

// ---------------------------------------------------------------------------
// The same pass with the other colour staged in shared memory by bulk copies.
// A CTA owns a column of one instance -- pair rows [y0, y0 + BY) of every
// colour site of the row (hx = Lx/2 a power of two, BY hx <= 256 threads) --
// and marches along z over its share of the (column, z) planes, so that each
// other-colour plane tile (rows y0 - 1 .. y0 + BY, wrapped in y) is copied
// once and serves the planes z - 1, z and z + 1.  A ring of four tiles holds
// z - 1, z, z + 1 while z + 2 is in flight; the own pairs of the next plane
// are copied into a second ring of two.  Results go straight to global
// memory (a site is read and written by its own thread only).
// ---------------------------------------------------------------------------
struct TileArgs {
    uint32_t by;                 // pair rows per tile
    uint32_t hx_shift;           // log2(hx)
    uint32_t nyb;                // column blocks per instance (Ly/2 / by)
    uint32_t ncol;               // columns over all instances
    uint64_t units;              // ncol * Lz planes
};

constexpr uint64_t kBulkWaitNs = 1000000000ull;   // 1 s

template <bool AXZ, bool SW>
__global__ void __launch_bounds__(256, 3) checker_pair_tiled_kernel(PairArgs a, TileArgs t, int colour, int hsel,
                                                                    int pass)
{
    int hd = -1;
    if (SW && !sweep_gate(a.sw, a.step, hd)) return;
    const bool h2 = SW && hd == 1;
    if (SW && hd >= 0) hsel = hd;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_abort;
    const uint32_t hx = a.hx, by = t.by, Ly2 = a.Ly2, Lz = a.Lz;
    const uint32_t to = (by + 2) * hx;          // pairs of an other-colour tile
    const uint32_t tw = by * hx;                // pairs of an own tile
    ulonglong2 *oring = reinterpret_cast<ulonglong2 *>(smem);      // 4 x (lo to | hi to)
    ulonglong2 *wring = oring + 8 * to;                             // 2 x (lo tw | hi tw)
    uint64_t *bar = reinterpret_cast<uint64_t *>(wring + 4 * tw);  // 4 other + 2 own
    const uint32_t tid = threadIdx.x;
    const uint32_t ty = tid >> t.hx_shift, tx = tid & (hx - 1);
    const bool active = ty < by;
    if (tid == 0) {
        for (int i = 0; i < 6; ++i) mbar_init(bar + i, 1);
        mbar_init_fence();
        s_abort = 0;
    }
    __syncthreads();
    const uint32_t step = static_cast<uint32_t>(*a.step);
    const uint64_t u_begin = uint64_t(blockIdx.x) * t.units / gridDim.x;
    const uint64_t u_end = uint64_t(blockIdx.x + 1) * t.units / gridDim.x;
    const int other = 1 - colour;
    uint32_t n_o = 0, n_w = 0;       // tiles issued into each ring so far (uniform)
    uint32_t c_o = 0, c_w = 0;       // tiles consumed (uniform)
    bool ok = true;
    for (uint64_t u = u_begin; u < u_end && ok;) {
        const uint32_t col = static_cast<uint32_t>(u / Lz);
        const uint32_t za = static_cast<uint32_t>(u - uint64_t(col) * Lz);
        const uint32_t zb = static_cast<uint32_t>(min(uint64_t(Lz), za + (u_end - u)));
        const int inst = static_cast<int>(col / t.nyb);
        const uint32_t y0 = (col - uint32_t(inst) * t.nyb) * by;
        const ulonglong2 *gbase = pair_state(a) + int64_t(inst) * a.n_inst_sites;
        const ulonglong2 *go = gbase + (other ? a.nhalf : 0);
        ulonglong2 *gw = const_cast<ulonglong2 *>(gbase) + (colour ? a.nhalf : 0);
        // thread 0: copy tile rows y0 - 1 .. y0 + by of other-colour plane zz
        auto issue_other = [&](uint32_t zz) {
            const uint32_t slot = n_o & 3u;
            uint64_t *b = bar + slot;
            ulonglong2 *dlo = oring + slot * 2 * to, *dhi = dlo + to;
            mbar_arrive_expect_tx(b, 2u * to * 16u);
            uint32_t r = 0;
            while (r < by + 2) {
                const uint32_t row = (y0 + Ly2 - 1 + r) % Ly2;
                const uint32_t run = min(by + 2 - r, Ly2 - row);
                const uint32_t src = (zz * Ly2 + row) * hx;
                bulk_copy_g2s(dlo + r * hx, go + src, run * hx * 16u, b);
                bulk_copy_g2s(dhi + r * hx, go + a.npair + src, run * hx * 16u, b);
                r += run;
            }
            ++n_o;
        };
        auto issue_own = [&](uint32_t zz) {
            const uint32_t slot = n_w & 1u;
            uint64_t *b = bar + 4 + slot;
            ulonglong2 *dlo = wring + slot * 2 * tw, *dhi = dlo + tw;
            mbar_arrive_expect_tx(b, 2u * tw * 16u);
            const uint32_t src = (zz * Ly2 + y0) * hx;
            bulk_copy_g2s(dlo, gw + src, tw * 16u, b);
            bulk_copy_g2s(dhi, gw + a.npair + src, tw * 16u, b);
            ++n_w;
        };
        if (tid == 0) {
            fence_proxy_async_smem();
            issue_other(za == 0 ? Lz - 1 : za - 1);
            issue_other(za);
            issue_other(za + 1 == Lz ? 0 : za + 1);
            issue_own(za);
        } else {
            n_o += 3;
            n_w += 1;
        }
        for (uint32_t z = za; z < zb; ++z) {
            if (tid == 0) {
                fence_proxy_async_smem();
                if (z + 2 <= zb) issue_other((z + 2) % Lz);
                if (z + 1 < zb) issue_own(z + 1);
            } else {
                if (z + 2 <= zb) ++n_o;
                if (z + 1 < zb) ++n_w;
            }
            const PairSite p = make_site(a, inst, z, y0 + ty, tx, colour);
            f2 g1{0}, g2{0}, g3{0};
            if (active && a.noise) site_noise(a, p, step, pass, g1, g2, g3);
            // tiles of planes z - 1, z, z + 1 (other) and z (own)
            const uint32_t im = c_o, i0 = c_o + 1, ip = c_o + 2, iw = c_w;
            bool got = mbar_wait(bar + (im & 3u), (im >> 2) & 1u, kBulkWaitNs) &&
                       mbar_wait(bar + (i0 & 3u), (i0 >> 2) & 1u, kBulkWaitNs) &&
                       mbar_wait(bar + (ip & 3u), (ip >> 2) & 1u, kBulkWaitNs) &&
                       mbar_wait(bar + 4 + (iw & 1u), (iw >> 1) & 1u, kBulkWaitNs);
            if (!got) {
                atomicOr(a.health, kHealthTimeout);
                s_abort = 1;
            }
            if (got && active) {
                const ulonglong2 *Tm = oring + (im & 3u) * 2 * to, *T0 = oring + (i0 & 3u) * 2 * to,
                                 *Tp = oring + (ip & 3u) * 2 * to, *Tw = wring + (iw & 1u) * 2 * tw;
                f2 htx, hty, htz, h1x, h1y, h1z;
                const uint32_t r1 = (ty + 1) * hx;
                neighbour_sums(p, hx, Ly2, T0, T0 + to, Tp, Tp + to, Tm, Tm + to, r1, r1, r1, (ty + 2) * hx,
                               ty * hx, htx, hty, htz, h1x, h1y, h1z);
                const uint32_t qs = ty * hx + tx;
                const uint32_t q = (z * Ly2 + y0 + ty) * hx + tx;
                pair_finish<AXZ>(a, p, colour, hsel, h2, g1, g2, g3, htx, hty, htz, h1x, h1y, h1z, Tw[qs],
                                 Tw[tw + qs], gw, gw + a.npair, q);
            }
            ++c_o;
            ++c_w;
            __syncthreads();
            if (s_abort) {
                ok = false;
                break;
            }
        }
        if (ok) {
            c_o += 2;          // the segment's last two tiles served as planes z and z + 1 of its last plane
            u += zb - za;
        }
    }
    // after a time-out: let this CTA's copies in flight land before exiting
    if (!ok && tid == 0) {
        for (uint32_t i = c_o - 1; i < n_o; ++i) mbar_wait(bar + (i & 3u), (i >> 2) & 1u, kBulkWaitNs);
        for (uint32_t i = c_w - 1; i < n_w; ++i) mbar_wait(bar + 4 + (i & 1u), (i >> 1) & 1u, kBulkWaitNs);
    }
}

// ---------------------------------------------------------------------------
// Fused symmetric sweep (FP32 site pairs, two colours): the three colour
// passes of a time step -- colour 0 for dt/2, colour 1 for dt, colour 0 for
// dt/2 -- in one launch, as a wavefront along z (temporal blocking), so that
// the state crosses HBM about once a step instead of three times.
//
// A cluster of C CTAs owns one z segment [z0, z1) of one instance; CTA r of
// the cluster owns pair rows [r R, r R + R) of every plane (C R = Ly/2), one
// pair column a thread, a third of the threads per pass.  At wavefront step
// t, with p0 = z0 - 2 + t, the CTA runs
//   pass 0 (colour 0, dt/2) on plane p0 + 2    (ahead, see below),
//   pass 1 (colour 1, dt)   on plane p0 - 2,
//   pass 2 (colour 0, dt/2) on plane p0 - 4.
// A pass on plane P needs the previous pass on P - 1, P and P + 1; with a lag
// of two planes those finished at earlier steps, so one cluster barrier a
// step orders everything.  Pass 0 reads only the state at the start of the
// step, so the pass-0 threads run the next step's plane while the other
// threads finish the current one.  The CTA's rows of the planes in flight
// live in shared memory: rings of 9 colour-1 and 8 colour-0 plane tiles,
// filled by bulk copies two steps ahead (the colour-1 halo rows y0 - 1 and
// y0 + R that pass 0 needs come with them, from global memory).  Passes 1 and
// 2 read the halo rows -- results of the neighbouring CTAs' earlier passes --
// from those CTAs' shared memory.  Pass 0 runs on planes z0 - 2 .. z1 + 1 and
// pass 1 on z0 - 1 .. z1, so that pass 2 has all it needs on z0 .. z1 - 1:
// neighbouring segments recompute two planes each side, which needs the
// input state unchanged while they run, so the kernel reads one state buffer
// and writes the other (and the last CTA to finish flips *cur).  Every site
// gets the same inputs, noise and arithmetic as in the three separate passes,
// so the spins are bitwise those of checker_pair_kernel.
// ---------------------------------------------------------------------------
struct SweepShape {
    uint32_t R = 0, C = 0;       // pair rows per CTA, CTAs per cluster (C R = Ly/2); C == 0: not offered
    uint32_t nseg = 1;           // z segments per instance
    uint32_t threads = 0;        // 3 R hx
    size_t smem = 0;
};

struct SweepArgs {
    uint32_t R, nseg;
    unsigned *done;              // CTAs finished; the last one flips *cur and clears this
    uint32_t ctas;
    int *cur;                    // writable view of PairArgs::cur
};

constexpr int kSwD1 = 9, kSwD0 = 8, kSwDH = 3;

inline size_t sweep_smem_bytes(uint32_t RH, uint32_t hx)
{
    return size_t(2u * (kSwD1 + kSwD0) * RH + 2u * kSwDH * 2u * hx) * 16u + 3 * sizeof(uint64_t);
}

__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// 16-byte loads from this CTA's shared memory and from a peer CTA's
// (distributed shared memory), by 32-bit shared-window addresses
__device__ __forceinline__ ulonglong2 lds16(uint32_t addr)
{
    ulonglong2 v;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
    return v;
}
__device__ __forceinline__ ulonglong2 ldsc16(uint32_t addr)
{
    ulonglong2 v;
    asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts16(uint32_t addr, ulonglong2 v)
{
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(v.x), "l"(v.y) : "memory");
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

template <bool AXZ>
__global__ void __launch_bounds__(768, 1) checker_sweep_kernel(PairArgs a, SweepArgs w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t hx = a.hx, Ly2 = a.Ly2, Lz = a.Lz, R = w.R, RH = R * hx;
    ulonglong2 *c1 = reinterpret_cast<ulonglong2 *>(smem);      // [kSwD1][lo RH | hi RH]
    ulonglong2 *c0 = c1 + 2u * kSwD1 * RH;                        // [kSwD0][lo RH | hi RH]
    ulonglong2 *hl = c0 + 2u * kSwD0 * RH;                        // [kSwDH][lo: y0-1, y0+R | hi: y0-1, y0+R]
    uint64_t *bar = reinterpret_cast<uint64_t *>(hl + 2u * kSwDH * 2u * hx);
    __shared__ int s_late;

    const uint32_t C = gridDim.x, rank = blockIdx.x, seg = blockIdx.y, inst = blockIdx.z;
    const uint32_t y0 = rank * R;
    const int z0 = static_cast<int>(uint64_t(seg) * Lz / w.nseg), z1 = static_cast<int>(uint64_t(seg + 1) * Lz / w.nseg);
    const int Z = z1 - z0, last_batch = Z + 3;
    const int cur = *a.cur;
    const ulonglong2 *in = (cur ? a.S1 : a.S) + int64_t(inst) * a.n_inst_sites;
    ulonglong2 *out = (cur ? a.S : a.S1) + int64_t(inst) * a.n_inst_sites;
    const ulonglong2 *in0 = in, *in1 = in + a.nhalf;             // colour 0 / 1, lo plane (hi at + npair)

    auto zwrap = [&](int p) {                                    // p in [-Lz, 2 Lz)
        return static_cast<uint32_t>(p < 0 ? p + static_cast<int>(Lz) : (p >= static_cast<int>(Lz) ? p - static_cast<int>(Lz) : p));
    };
    auto tile1 = [&](int p) { return c1 + 2u * RH * (static_cast<uint32_t>(p - (z0 - 3)) % kSwD1); };
    auto tile0 = [&](int p) { return c0 + 2u * RH * (static_cast<uint32_t>(p - (z0 - 3)) % kSwD0); };

    // batch u: the CTA's colour-1 rows of plane p0(u) + 1 and colour-0 rows of
    // p0(u), and the colour-1 halo rows at p0(u); batch 0 also brings the
    // colour-1 rows of p0(0) - 1 and p0(0)
    auto issue = [&](int u) {
        const int p0 = z0 - 2 + u;
        uint64_t *b = bar + (u % 3);
        const uint32_t rb = RH * 16u, hb = hx * 16u;
        mbar_arrive_expect_tx(b, (u == 0 ? 8u : 4u) * rb + 4u * hb);
        auto rows = [&](const ulonglong2 *src, int p, ulonglong2 *dst) {
            const uint32_t q = (zwrap(p) * Ly2 + y0) * hx;
            bulk_copy_g2s(dst, src + q, rb, b);
            bulk_copy_g2s(dst + RH, src + a.npair + q, rb, b);
        };
        if (u == 0) {
            rows(in1, p0 - 1, tile1(p0 - 1));
            rows(in1, p0, tile1(p0));
        }
        rows(in1, p0 + 1, tile1(p0 + 1));
        rows(in0, p0, tile0(p0));
        ulonglong2 *h = hl + (u % kSwDH) * 4u * hx;
        const uint32_t zz = zwrap(p0);
        const uint32_t qm = (zz * Ly2 + (y0 + Ly2 - 1) % Ly2) * hx, qp = (zz * Ly2 + (y0 + R) % Ly2) * hx;
        bulk_copy_g2s(h, in1 + qm, hb, b);
        bulk_copy_g2s(h + hx, in1 + qp, hb, b);
        bulk_copy_g2s(h + 2u * hx, in1 + a.npair + qm, hb, b);
        bulk_copy_g2s(h + 3u * hx, in1 + a.npair + qp, hb, b);
    };

    // ---- this thread: pass g on pair column jcol (row r, colour site kx) ----
    const uint32_t tid = threadIdx.x;
    const uint32_t g = tid / RH, jcol = tid - g * RH;
    const uint32_t r = jcol / hx, kx = jcol - r * hx, y2 = y0 + r;
    const int colour = g == 1 ? 1 : 0;
    const uint32_t kxp = kx + 1 == hx ? 0 : kx + 1, kxm = kx == 0 ? hx - 1 : kx - 1;
    const uint32_t step = static_cast<uint32_t>(*a.step);
    const uint32_t ig = a.inst_base + inst;
    const uint32_t peer_up = rank + 1 == C ? 0 : rank + 1, peer_dn = rank == 0 ? C - 1 : rank - 1;
    // shared-window byte addresses: own ring (this pass's colour), other ring, halo slots
    const uint32_t tileB = 2u * RH * 16u, hiB = RH * 16u;
    const uint32_t own_base = smem_u32(colour ? c1 : c0), oth_base = smem_u32(colour ? c0 : c1);
    const uint32_t Down = colour ? kSwD1 : kSwD0, Doth = colour ? kSwD0 : kSwD1;
    const uint32_t halo_base = smem_u32(hl);
    const uint32_t colB = jcol * 16u;
    // invariants of the site pair's noise counter and TTM cell
    const uint32_t atom_row = y2 * a.Lx + 2 * kx, plane_atoms = a.Ly * a.Lx;
    const uint32_t cell_inst = static_cast<uint32_t>(a.cell0 + static_cast<int>(inst) * a.cstride);
    auto cc = [](uint32_t v, uint32_t n, const FastDiv &d, int sh) { return sh >= 0 ? v >> sh : fast_div(v * n, d); };
    const uint32_t cyA = cc(y2, a.ncy, a.dLy, a.shy), cyB = cc(y2 + Ly2, a.ncy, a.dLy, a.shy);
    const uint32_t cx0 = cc(2 * kx, a.ncx, a.dLx, a.shx), cx1 = cc(2 * kx + 1, a.ncx, a.dLx, a.shx);
    const int hsel = colour;
    const uint32_t par_flip = Ly2 & 1u;

    // prepared for the next pass of this thread (independent of any spin):
    // its plane, noise directions and the noise amplitudes of both species
    struct Prep {
        int P;
        uint32_t zP, parA;
        uint32_t so, sm, s0, sp;     // ring slots: own tile of P; other tiles of P - 1, P, P + 1
        f2 g1, g2, g3;
        float sA[2], sB[2];
    };
    // ring-slot byte offsets advance one tile a step (a pass moves one plane)
    const uint32_t own_wrap = Down * tileB, oth_wrap = Doth * tileB;
    auto adv = [](uint32_t v, uint32_t step_b, uint32_t wrap) { v += step_b; return v == wrap ? 0u : v; };
    auto prepare = [&](int t, Prep &q, bool fresh) {
        q.P = z0 - 2 + t - 2 * static_cast<int>(g);
        q.zP = zwrap(q.P);
        if (fresh) {
            const uint32_t rel = static_cast<uint32_t>(q.P - (z0 - 3));
            q.so = (rel % Down) * tileB;
            q.sm = ((rel - 1) % Doth) * tileB;
            q.s0 = (rel % Doth) * tileB;
            q.sp = ((rel + 1) % Doth) * tileB;
        } else {
            q.so = adv(q.so, tileB, own_wrap);
            q.sm = adv(q.sm, tileB, oth_wrap);
            q.s0 = adv(q.s0, tileB, oth_wrap);
            q.sp = adv(q.sp, tileB, oth_wrap);
        }
        q.parA = (y2 + q.zP + uint32_t(colour)) & 1u;
        const uint32_t parB = q.parA ^ par_flip;
        q.g1 = q.g2 = q.g3 = f2{0};
        q.sA[0] = q.sA[1] = q.sB[0] = q.sB[1] = 0.0f;
        if (a.noise) {
            const uint32_t atomA = q.zP * plane_atoms + atom_row + q.parA;
            const uint32_t atomB = atomA + Ly2 * a.Lx + parB - q.parA;
            pair_noise(u32x4{atomA, step, g, ig}, u32x4{atomB, step, g, ig}, a.rk, a.k, q.g1, q.g2, q.g3);
            int cA, cB;
            if (a.cell_formula) {
                const uint32_t cz = cc(q.zP, a.ncz, a.dLz, a.shz);
                const uint32_t base = cell_inst + cz * a.ncy * a.ncx;
                cA = static_cast<int>(base + cyA * a.ncx + (q.parA ? cx1 : cx0));
                cB = static_cast<int>(base + cyB * a.ncx + (parB ? cx1 : cx0));
            } else {
                const uint32_t slotA = uint32_t(colour) * a.nhalf + (q.zP * a.Ly + y2) * hx + kx;
                const int *cell = a.cell + int64_t(inst) * a.n_inst_sites;
                cA = cell[slotA];
                cB = cell[slotA + Ly2 * hx];
            }
            const float *sg = a.sigma + hsel;
            q.sA[0] = __ldg(sg + cA * 4);
            q.sA[1] = __ldg(sg + cA * 4 + 2);
            q.sB[0] = __ldg(sg + cB * 4);
            q.sB[1] = __ldg(sg + cB * 4 + 2);
        }
    };

    auto ldpair = [&](uint32_t lo) {        // lo and hi words of a pair in this CTA's shared memory
        const ulonglong2 l = lds16(lo), h = lds16(lo + hiB);
        return Pair4{f2{l.x}, f2{l.y}, f2{h.x}, f2{h.y}};
    };
    auto ldpeer = [&](uint32_t lo, uint32_t peer) {
        const ulonglong2 l = ldsc16(peer_addr(lo, peer)), h = ldsc16(peer_addr(lo + hiB, peer));
        return Pair4{f2{l.x}, f2{l.y}, f2{h.x}, f2{h.y}};
    };

    // the pass itself, from prepared data
    auto compute = [&](int t, const Prep &q) {
        const int P = q.P;
        const uint32_t Wt = own_base + q.so;
        const uint32_t Om = oth_base + q.sm, O0 = oth_base + q.s0, Op = oth_base + q.sp;
        f2 htx{0}, hty{0}, htz{0}, h1x{0}, h1y{0}, h1z{0};
        // sum order z+1, z-1, y+1, y-1, x, x' (that of checker_pair_kernel)
        add_neighbour(ldpair(Op + colB), htx, hty, htz, h1x, h1y, h1z);
        add_neighbour(ldpair(Om + colB), htx, hty, htz, h1x, h1y, h1z);
        {
            Pair4 n;
            if (r + 1 < R) {
                n = ldpair(O0 + colB + hx * 16u);
            } else if (g == 0) {
                const uint32_t h = halo_base + (static_cast<uint32_t>(t) % kSwDH) * 64u * hx + (hx + kx) * 16u;
                const ulonglong2 l = lds16(h), hh = lds16(h + 32u * hx);
                n = Pair4{f2{l.x}, f2{l.y}, f2{hh.x}, f2{hh.y}};
            } else {
                n = ldpeer(O0 + kx * 16u, peer_up);                  // row 0 of the CTA above
            }
            if (y2 + 1 == Ly2) n = swap_lanes(n);
            add_neighbour(n, htx, hty, htz, h1x, h1y, h1z);
        }
        {
            Pair4 n;
            if (r > 0) {
                n = ldpair(O0 + colB - hx * 16u);
            } else if (g == 0) {
                const uint32_t h = halo_base + (static_cast<uint32_t>(t) % kSwDH) * 64u * hx + kx * 16u;
                const ulonglong2 l = lds16(h), hh = lds16(h + 32u * hx);
                n = Pair4{f2{l.x}, f2{l.y}, f2{hh.x}, f2{hh.y}};
            } else {
                n = ldpeer(O0 + ((R - 1) * hx + kx) * 16u, peer_dn);  // last row of the CTA below
            }
            if (y2 == 0) n = swap_lanes(n);
            add_neighbour(n, htx, hty, htz, h1x, h1y, h1z);
        }
        add_neighbour(ldpair(O0 + colB), htx, hty, htz, h1x, h1y, h1z);
        const uint32_t rowB = O0 + r * hx * 16u;
        const uint32_t parB = q.parA ^ par_flip;
        if (q.parA == parB) {
            add_neighbour(ldpair(rowB + (q.parA ? kxp : kxm) * 16u), htx, hty, htz, h1x, h1y, h1z);
        } else {
            const Pair4 Pp = ldpair(rowB + kxp * 16u), M = ldpair(rowB + kxm * 16u);
            const Pair4 &LA = q.parA ? Pp : M, &LB = q.parA ? M : Pp;
            add_neighbour(Pair4{f2_mix(LA.x, LB.x), f2_mix(LA.y, LB.y), f2_mix(LA.z, LB.z), f2_mix(LA.w, LB.w)}, htx,
                          hty, htz, h1x, h1y, h1z);
        }
        const ulonglong2 olo = lds16(Wt + colB), ohi = lds16(Wt + colB + hiB);
        f2 sx{olo.x}, sy{olo.y}, sz{ohi.x};
        const f2 wv{ohi.y};
        f2 sig{0};
        if (a.noise) {
            float wA, wB;
            f2_split(wv, wA, wB);
            sig = f2_make(wA != 0.0f ? q.sA[1] : q.sA[0], wB != 0.0f ? q.sB[1] : q.sB[0]);
        }
        // the constants are made for dt/2; pass 1 runs for dt (the step-length
        // terms doubled, exactly as the separate pass's own constants)
        pair_update<AXZ>(sx, sy, sz, htx, hty, htz, h1x, h1y, h1z, wv, a.noise != 0, sig, q.g1, q.g2, q.g3, a.k,
                         g == 1);
        float sA, sB;
        f2_split(sx + sy + sz, sA, sB);
        if (!isfinite(sA) || !isfinite(sB)) atomicOr(a.health, kHealthNonFinite);
        // the result replaces the pair in its tile: for the later passes and
        // the neighbouring CTAs (passes 0 and 1), and for the bulk store of
        // the finished plane (passes 1 and 2)
        sts16(Wt + colB, ulonglong2{sx.v, sy.v});
        sts16(Wt + colB + hiB, ulonglong2{sz.v, ohi.y});
    };
    // thread 0, after the barrier that follows step t: the CTA's rows of the
    // planes finished in step t -- colour 1 of p0(t) - 2 (pass 1) and colour 0
    // of p0(t) - 4 (pass 2) -- to the output buffer, by bulk copies (no
    // generic global stores, so the barriers' release orders shared memory
    // only); the groups are waited for before their tiles are refilled
    auto store_finished = [&](int t) {
        bool any = false;
        const int P1 = z0 - 4 + t, P2 = z0 - 6 + t;
        if (t >= 3 && P1 >= z0 && P1 < z1) {
            const ulonglong2 *src = tile1(P1);
            ulonglong2 *dst = out + a.nhalf + (zwrap(P1) * Ly2 + y0) * hx;
            bulk_copy_s2g(dst, src, RH * 16u);
            bulk_copy_s2g(dst + a.npair, src + RH, RH * 16u);
            any = true;
        }
        if (t >= 6 && P2 >= z0 && P2 < z1) {
            const ulonglong2 *src = tile0(P2);
            ulonglong2 *dst = out + (zwrap(P2) * Ly2 + y0) * hx;
            bulk_copy_s2g(dst, src, RH * 16u);
            bulk_copy_s2g(dst + a.npair, src + RH, RH * 16u);
            any = true;
        }
        if (any) bulk_commit();
    };

    auto wait_batch = [&](int u) {
        if (!mbar_wait(bar + (u % 3), static_cast<uint32_t>(u / 3) & 1u, kBulkWaitNs)) {
            atomicOr(a.health, kHealthTimeout);
            s_late = 1;
        }
    };

    if (tid == 0) {
        s_late = 0;
        for (int i = 0; i < 3; ++i) mbar_init(bar + i, 1);
        mbar_init_fence();
        issue(0);
        if (1 <= last_batch) issue(1);
    }
    // the first step of each pass: pass 0 runs step 0 before the loop (and
    // step t + 1 in iteration t), pass 1 from step 3, pass 2 from step 6
    const int first = g == 0 ? 0 : (g == 1 ? 3 : 6);
    const int lastt = g == 0 ? last_batch : (g == 1 ? Z + 4 : Z + 5);
    Prep q;
    prepare(first, q, true);
    __syncthreads();
    if (g == 0) {
        wait_batch(0);
        compute(0, q);
        if (1 <= lastt) prepare(1, q, false);
    }
    cluster_arrive();
    const int T = Z + 6;
    for (int t = 0; t < T; ++t) {
        cluster_wait();                      // every CTA of the cluster finished step t - 1
        if (tid == 0) {
            fence_proxy_async_smem();        // the threads' tile writes, before the bulk engine reads them
            if (t >= 1) store_finished(t - 1);
            // tiles refilled by this batch were stored (if at all) at least
            // two steps ago: let all but the newest store group finish reading
            bulk_wait_read<1>();
            if (t + 2 <= last_batch) issue(t + 2);
        }
        const int mine = g == 0 ? t + 1 : t; // the step this thread's pass runs in this iteration
        const bool run = mine >= first && mine <= lastt;
        if (run) {
            if (g == 0) wait_batch(mine);
            compute(mine, q);
        }
        cluster_arrive();
        // the next step's noise and amplitudes while the barrier completes
        if (run && mine + 1 <= lastt) prepare(mine + 1, q, false);
    }
    cluster_wait();                          // no CTA leaves while a peer may still read its tiles
    __syncthreads();
    if (tid == 0) {
        fence_proxy_async_smem();
        store_finished(T - 1);
        bulk_wait_all();                     // the output is written before the flip below
        // after a wait that ran out, let the copies still in flight land
        // (again bounded) before the CTA's shared memory goes away
        if (s_late)
            for (int u = max(0, last_batch - 2); u <= last_batch; ++u)
                mbar_wait(bar + (u % 3), static_cast<uint32_t>(u / 3) & 1u, kBulkWaitNs);
        __threadfence();
        if (atomicAdd(w.done, 1u) == w.ctas - 1) {
            *w.cur = 1 - cur;
            *w.done = 0u;
            __threadfence();
        }
    }
}

// Observables of the pair layout: the same per-species partial sums, block
// by block, as the general observable kernel.  Per site, in FP32 and tesla
// (the spins are FP32): the unit-free terms s, s.h, (s.n)^2, B.s,
// |s x B_tot|^2, s.B_tot (h the exchange field, B_tot = h + kappa (s.n) n + B).
// Every sum over sites is FP64: each site's terms are converted exactly to
// double and added to FP64 accumulators per species (species-1 sums by a
// fused multiply-add with the 0/1 species flag, species 0 as the difference
// from the all-site sum); the block then reduces the threads' accumulators in
// a fixed order and scales them by mu and K of the species.
struct PairObsArgs {
    const int *obs_block_inst;
    const DevInstance *inst;
    double *obs_partial;
    int obs_blocks;
    int sample_every;
    double mu[TTS_MAX_SPECIES], K[TTS_MAX_SPECIES];
};

// Factor of observable field f (12 per species): 1 for the count and the sums
// of s; -mu/2 (exchange), -K, -mu (Zeeman), mu^2 (|s x H|^2), mu (s.H).
__device__ __forceinline__ double obs_scale(const PairObsArgs &o, int f)
{
    const int sp = f >= 12 ? 1 : 0, r = f - 12 * sp;
    const double mu = sp ? o.mu[1] : o.mu[0], K = sp ? o.K[1] : o.K[0];
    switch (r) {
    case 7: return -0.5 * mu;
    case 8: return -K;
    case 9: return -mu;
    case 10: return mu * mu;
    case 11: return mu;
    default: return 1.0;
    }
}

constexpr int kObsTerms = 8;

// Compensated sums.  A pair (s, c) of floats stands for s + c; adding x
// replaces s by the rounded s + x and adds that addition's rounding error,
// computed exactly by TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2), to c.  Only
// the additions into c round, each by at most eps = 2^-24 times the c it
// makes, and a c that is d additions deep holds at most d eps times the sum
// of the |terms| below it.  A block partial is d <= 12 deep on every path
// (four pairs a lane, the two lanes, four threads, five shuffle levels), so
// it is within 144 eps^2 sum|x| < 2^-40 sum|x| of the exact sum of its 1024
// FP32 site terms (FP64 accumulation in the same order would guarantee
// 12 * 2^-53 sum|x|), far below the terms' own FP32 rounding (up to
// eps sum|x|).  Block partials are summed in FP64.
struct Comp2 {                 // both lanes of an f2
    f2 s, c;
};
__device__ __forceinline__ void comp_add(Comp2 &a, f2 x)
{
    const f2 t = a.s + x;
    const f2 xv = t - a.s;                 // the part of x that reached t
    const f2 e = (a.s - (t - xv)) + (x - xv);
    a.s = t;
    a.c = a.c + e;
}
struct Comp1 {
    float s, c;
};
__device__ __forceinline__ Comp1 comp_sum(Comp1 a, Comp1 b)
{
    const float t = __fadd_rn(a.s, b.s);
    const float bv = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bv)), __fsub_rn(b.s, bv));
    return Comp1{t, __fadd_rn(__fadd_rn(a.c, b.c), e)};
}
__device__ __forceinline__ Comp1 comp_lanes(const Comp2 &a)
{
    float sA, sB, cA, cB;
    f2_split(a.s, sA, sB);
    f2_split(a.c, cA, cB);
    return comp_sum(Comp1{sA, cA}, Comp1{sB, cB});
}

// Sum NF compensated values over the kObsBlock threads: shared memory, then
// warp w sums the fields f = w, w + 4, ... (each lane four threads' values,
// then a five-level shuffle tree), in a fixed order.  Field f's sum, as a
// double, times scale(f) is stored at out[f] by thread f (the FP64 work of
// all fields in one warp instruction each: the FP64 pipe takes 16 clocks a
// warp instruction however few lanes are active).
template <int NF, typename Scale>
__device__ __forceinline__ void block_sum_comp(const Comp1 (&v)[NF], Scale scale, double *out)
{
    static_assert(kObsBlock == 128 && NF <= 32, "four warps of 32, one lane a field");
    __shared__ float shs[NF][kObsBlock], shc[NF][kObsBlock];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        shs[f][threadIdx.x] = v[f].s;
        shc[f][threadIdx.x] = v[f].c;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int f = warp; f < NF; f += kObsBlock / 32) {
        auto at = [&](int i) { return Comp1{shs[f][i], shc[f][i]}; };
        Comp1 x = comp_sum(comp_sum(at(lane), at(lane + 32)), comp_sum(at(lane + 64), at(lane + 96)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            x = comp_sum(x, Comp1{__shfl_down_sync(0xffffffffu, x.s, o), __shfl_down_sync(0xffffffffu, x.c, o)});
        __syncwarp();
        if (lane == 0) {                // row f is read by this warp only, and no longer
            shs[f][0] = x.s;
            shc[f][0] = x.c;
        }
    }
    __syncthreads();
    if (threadIdx.x < NF) out[threadIdx.x] = (double(shs[threadIdx.x][0]) + double(shc[threadIdx.x][0])) * scale(threadIdx.x);
    __syncthreads();
}

__global__ void __launch_bounds__(kObsBlock) checker_pair_obs_kernel(PairArgs a, PairObsArgs o, int mode)
{
    const int64_t step = *a.step;
    if (mode == 0 && (o.sample_every <= 0 || (step + 1) % o.sample_every != 0)) return;
    const uint32_t hx = a.hx, Ly2 = a.Ly2, Lz = a.Lz;
    const PairConsts &k = a.k;
    for (int blk = blockIdx.x; blk < o.obs_blocks; blk += gridDim.x) {
        const int inst = o.obs_block_inst[blk];
        const uint32_t local = static_cast<uint32_t>(blk - o.inst[inst].obs_block_begin);
        Comp2 all[kObsTerms], one[kObsTerms];
#pragma unroll
        for (int t = 0; t < kObsTerms; ++t) all[t] = one[t] = Comp2{f2{0}, f2{0}};
        int n_all = 0, n_one = 0;
        const ulonglong2 *base = pair_state(a) + int64_t(inst) * a.n_inst_sites;
        for (int j = 0; j < kObsSpan / 2 / kObsBlock; ++j) {
            const uint32_t P = local * (kObsSpan / 2) + threadIdx.x + uint32_t(j) * kObsBlock;
            if (P >= 2 * a.npair) break;
            const int colour = P >= a.npair ? 1 : 0;
            const uint32_t q = P - uint32_t(colour) * a.npair;
            const uint32_t zy = q / hx, kx = q - zy * hx;
            const uint32_t z = zy / Ly2, y2 = zy - z * Ly2;
            const PairSite ps = make_site(a, inst, z, y2, kx, colour);
            const ulonglong2 *Olo = base + (colour ? 0 : a.nhalf), *Ohi = Olo + a.npair;
            const ulonglong2 *Wlo = base + (colour ? a.nhalf : 0), *Whi = Wlo + a.npair;
            const uint32_t zp = (z + 1 == Lz) ? 0 : z + 1, zm = (z == 0) ? Lz - 1 : z - 1;
            const uint32_t yp = (y2 + 1 == Ly2) ? 0 : y2 + 1, ym = (y2 == 0) ? Ly2 - 1 : y2 - 1;
            f2 htx, hty, htz, h1x, h1y, h1z;
            neighbour_sums(ps, hx, Ly2, Olo, Ohi, Olo, Ohi, Olo, Ohi, (zp * Ly2 + y2) * hx, (zm * Ly2 + y2) * hx,
                           zy * hx, (z * Ly2 + yp) * hx, (z * Ly2 + ym) * hx, htx, hty, htz, h1x, h1y, h1z);
            const ulonglong2 lo = Wlo[q], hi = Whi[q];
            const f2 sx{lo.x}, sy{lo.y}, sz{hi.x}, w{hi.y};
            const f2 J0 = fma2(w, k.J0d, k.J0c), dJ = fma2(w, k.dJd, k.dJc), kap = fma2(w, k.kd, k.kc);
            const f2 hX = fma2(J0, htx, dJ * h1x), hY = fma2(J0, hty, dJ * h1y), hZ = fma2(J0, htz, dJ * h1z);
            const f2 sn = fma2(sz, k.nz, fma2(sy, k.ny, sx * k.nx));
            const f2 ka = kap * sn;
            const f2 Bx = fma2(ka, k.nx, hX + k.Bx), By = fma2(ka, k.ny, hY + k.By), Bz = fma2(ka, k.nz, hZ + k.Bz);
            const f2 cx = sy * Bz - sz * By, cy = sz * Bx - sx * Bz, cz = sx * By - sy * Bx;
            const f2 term[kObsTerms] = {sx,
                                        sy,
                                        sz,
                                        fma2(sz, hZ, fma2(sy, hY, sx * hX)),
                                        sn * sn,
                                        fma2(sz, k.Bz, fma2(sy, k.By, sx * k.Bx)),
                                        fma2(cz, cz, fma2(cy, cy, cx * cx)),
                                        fma2(sz, Bz, fma2(sy, By, sx * Bx))};
            float wA, wB;
            f2_split(w, wA, wB);
            n_all += 2;
            n_one += (wA != 0.0f) + (wB != 0.0f);
#pragma unroll
            for (int t = 0; t < kObsTerms; ++t) {
                comp_add(all[t], term[t]);
                comp_add(one[t], w * term[t]);        // exact: w is 0 or 1
            }
        }
        Comp1 acc[kObsFields];
#pragma unroll
        for (int f = 0; f < kObsFields; ++f) acc[f] = Comp1{0.0f, 0.0f};
        acc[0] = Comp1{float(n_all - n_one), 0.0f};   // counts below 2^24: exact
        acc[12] = Comp1{float(n_one), 0.0f};
#pragma unroll
        for (int t = 0; t < kObsTerms; ++t) {
            // species 0: all sites minus species 1, term by term
            const Comp1 v1 = comp_lanes(one[t]);
            const Comp1 v0 = comp_sum(comp_lanes(all[t]), Comp1{-v1.s, -v1.c});
            const int f = t < 3 ? 1 + t : 4 + t;       // s -> 1..3; the five others -> 7..11
            acc[f] = v0;
            acc[12 + f] = v1;
        }
        block_sum_comp<kObsFields>(acc, [&](int f) { return obs_scale(o, f); },
                                   o.obs_partial + int64_t(blk) * kObsFields);
    }
}

// pair planes <-> general SoA.  One thread per pair; general slot of a site
// within its instance: colour * nhalf + (z Ly + y) hx + kx.
__global__ void pair_to_general_kernel(const float4 *S0, const float4 *S1, const int *cur, float *sx, float *sy,
                                       float *sz, int64_t npairs, uint32_t hx, uint32_t Ly2, uint32_t npair,
                                       const int64_t *step, int sample_every, int conditional)
{
    if (conditional && (sample_every <= 0 || (*step + 1) % sample_every != 0)) return;
    const float4 *__restrict__ S = *cur ? S1 : S0;
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= npairs) return;
    const int64_t block = g / npair;              // (instance, colour) block
    const uint32_t q = static_cast<uint32_t>(g - block * npair);
    const int64_t site0 = block * int64_t(2 * npair);   // first general slot of the block
    const uint32_t zy = q / hx, kx = q - zy * hx;
    const uint32_t z = zy / Ly2, y2 = zy - z * Ly2;
    const int64_t iA = site0 + (int64_t(z) * 2 * Ly2 + y2) * hx + kx;
    const int64_t iB = iA + int64_t(Ly2) * hx;
    const float4 lo = S[site0 + q], hi = S[site0 + npair + q];
    sx[iA] = lo.x;
    sx[iB] = lo.y;
    sy[iA] = lo.z;
    sy[iB] = lo.w;
    sz[iA] = hi.x;
    sz[iB] = hi.y;
}

__global__ void pair_from_general_kernel(float4 *S0, float4 *S1, const int *cur, const float *__restrict__ sx,
                                         const float *__restrict__ sy, const float *__restrict__ sz,
                                         const uint8_t *__restrict__ spc, int64_t npairs, uint32_t hx, uint32_t Ly2,
                                         uint32_t npair)
{
    float4 *S = *cur ? S1 : S0;
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= npairs) return;
    const int64_t block = g / npair;
    const uint32_t q = static_cast<uint32_t>(g - block * npair);
    const int64_t site0 = block * int64_t(2 * npair);
    const uint32_t zy = q / hx, kx = q - zy * hx;
    const uint32_t z = zy / Ly2, y2 = zy - z * Ly2;
    const int64_t iA = site0 + (int64_t(z) * 2 * Ly2 + y2) * hx + kx;
    const int64_t iB = iA + int64_t(Ly2) * hx;
    S[site0 + q] = make_float4(sx[iA], sx[iB], sy[iA], sy[iB]);
    S[site0 + npair + q] = make_float4(sz[iA], sz[iB], spc[iA] ? 1.0f : 0.0f, spc[iB] ? 1.0f : 0.0f);
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
    int merged;                          // merged (leapfrog) sweep
    TtmParams tp;
    PairConsts pk;                       // FP32: constants of the pair update for h = dt/2
    PhiloxRoundKeys rk;
    // bath trajectory of the current chunk of steps, per instance: noise table
    // [species][h] of each step and (T_e, T_l) after it
    R *traj_sig;
    double *traj_T;
    int traj_cap;                        // steps per instance slot
    // merged sweep across chunks of one call: colour 0 open at the end of a chunk
    int *open_state;                     // per instance
    int first_chunk, last_chunk;
};

// The six nearest neighbours (periodic simple-cubic) of canonical atom `at` of
// an instance of L cells.
__device__ __forceinline__ void resident_nbrs(uint32_t at, const ResInst &I, uint32_t nb[6])
{
    const int Lx = I.L[0], Ly = I.L[1], Lz = I.L[2];
    const uint32_t z = fast_div(at, I.divxy);
    const uint32_t rem = at - z * uint32_t(Lx * Ly);
    const uint32_t y = fast_div(rem, I.divx);
    const uint32_t x = rem - y * uint32_t(Lx);
    const uint32_t xp = x + 1 == uint32_t(Lx) ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
    const uint32_t yp = y + 1 == uint32_t(Ly) ? 0 : y + 1, ym = y == 0 ? Ly - 1 : y - 1;
    const uint32_t zp = z + 1 == uint32_t(Lz) ? 0 : z + 1, zm = z == 0 ? Lz - 1 : z - 1;
    nb[0] = (zp * Ly + y) * Lx + x;
    nb[1] = (zm * Ly + y) * Lx + x;
    nb[2] = (z * Ly + yp) * Lx + x;
    nb[3] = (z * Ly + ym) * Lx + x;
    nb[4] = (z * Ly + y) * Lx + xp;
    nb[5] = (z * Ly + y) * Lx + xm;
}

// Their spin sums: all and species-1 only.
template <typename R>
__device__ __forceinline__ void resident_sums(uint32_t at, const ResInst &I, const R *sx, const R *sy, const R *sz,
                                              const uint8_t *spc, R &htx, R &hty, R &htz, R &h1x, R &h1y, R &h1z)
{
    uint32_t nb[6];
    resident_nbrs(at, I, nb);
    htx = hty = htz = h1x = h1y = h1z = R(0);
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
}

// FP32 resident colour pass: two colour sites per thread on the packed f32x2
// update, entry j of the colour's first half with entry j of its second half
// (so that a warp's A lanes and B lanes each read consecutive entries); with
// an odd count the middle entry runs in both lanes and is stored once.
template <bool AXZ>
__device__ __forceinline__ void resident_pair_pass(const ResArgs<float> &a, const ResInst &I, float *sx, float *sy,
                                                   float *sz, const uint8_t *spc, int beg, int end, int64_t step,
                                                   int p, int hsel, const float (*sig_tab)[2])
{
    const int half = (end - beg + 1) >> 1;
    const bool noise = sig_tab[0][hsel] > 0.0f || sig_tab[1][hsel] > 0.0f;
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
        const int iA = beg + j, iB0 = iA + half, iB = iB0 < end ? iB0 : iA;
        const uint32_t atA = static_cast<uint32_t>(a.atom[I.slot_begin + iA]);
        const uint32_t atB = static_cast<uint32_t>(a.atom[I.slot_begin + iB]);
        f2 g1{0}, g2{0}, g3{0};
        if (noise)
            pair_noise(u32x4{atA, static_cast<uint32_t>(step), static_cast<uint32_t>(p), I.inst_global},
                       u32x4{atB, static_cast<uint32_t>(step), static_cast<uint32_t>(p), I.inst_global}, a.rk, a.pk,
                       g1, g2, g3);
        uint32_t nA[6], nB[6];
        resident_nbrs(atA, I, nA);
        resident_nbrs(atB, I, nB);
        f2 htx{0}, hty{0}, htz{0}, h1x{0}, h1y{0}, h1z{0};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const f2 vx = f2_make(sx[nA[k]], sx[nB[k]]);
            const f2 vy = f2_make(sy[nA[k]], sy[nB[k]]);
            const f2 vz = f2_make(sz[nA[k]], sz[nB[k]]);
            const f2 w = f2_make(spc[nA[k]] ? 1.0f : 0.0f, spc[nB[k]] ? 1.0f : 0.0f);
            htx = htx + vx;
            hty = hty + vy;
            htz = htz + vz;
            h1x = fma2(w, vx, h1x);
            h1y = fma2(w, vy, h1y);
            h1z = fma2(w, vz, h1z);
        }
        const int tA = spc[atA], tB = spc[atB];
        f2 px = f2_make(sx[atA], sx[atB]), py = f2_make(sy[atA], sy[atB]), pz = f2_make(sz[atA], sz[atB]);
        const f2 w = f2_make(tA ? 1.0f : 0.0f, tB ? 1.0f : 0.0f);
        pair_update<AXZ>(px, py, pz, htx, hty, htz, h1x, h1y, h1z, w, noise,
                         f2_make(sig_tab[tA][hsel], sig_tab[tB][hsel]), g1, g2, g3, a.pk, hsel == 1);
        float lx, hx_, ly, hy, lz, hz;
        f2_split(px, lx, hx_);
        f2_split(py, ly, hy);
        f2_split(pz, lz, hz);
        // same-colour sites are not neighbours: no other thread reads these until the pass ends
        sx[atA] = lx;
        sy[atA] = ly;
        sz[atA] = lz;
        if (iB != iA) {
            sx[atB] = hx_;
            sy[atB] = hy;
            sz[atB] = hz;
        }
    }
}

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

// Thread 0's FP64 work for one step, out of line so that it does not raise
// the register count of the spin loop: the noise table of step `step` from
// T_e (mode 0), or the one-cell TTM advance t_n -> t_n+1 (mode 1).
template <typename R>
__device__ __noinline__ void resident_bath(const ResArgs<R> &a, const DevInstance &D, int64_t step, int mode,
                                           double *T, double *deposited, R *sigma_out)
{
    if (mode == 0) {
        for (int t = 0; t < TTS_MAX_SPECIES; ++t)
            for (int hs = 0; hs < 2; ++hs) {
                double v = 0.0;
                if (t < a.nspecies && T[0] > 0.0 && a.spd[t].alpha > 0.0) {
                    const double h = hs ? a.dt : 0.5 * a.dt;
                    v = sqrt(2.0 * a.spd[t].alpha * kBoltzmann * T[0] / (kGyro * a.spd[t].mu * h));
                }
                sigma_out[t * 2 + hs] = static_cast<R>(v);
            }
        return;
    }
    if (a.tp.source == TTS_SOURCE_STEP_PROFILE) {
        const double tt = double(step + 1) * a.dt;
        T[0] = tt < D.prof_t1 ? D.prof_peak : (tt < D.prof_t2 ? 0.5 * D.prof_peak : a.tp.T0);
        T[1] = a.tp.T0;
        return;
    }
    double Te = T[0], Tl = T[1];
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
        *deposited += delta * src * D.cell_volume;
        Tl += delta * xch / a.tp.C_l;
        Te = sqrt(2.0 * (0.5 * a.tp.gamma_e * Te * Te + dE) / a.tp.gamma_e);
    }
    T[0] = Te;
    T[1] = Tl;
}

template <typename R, bool AXZ>
__global__ void __launch_bounds__(512, 1) resident_kernel(ResArgs<R> a, int64_t nsteps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    R *sx = reinterpret_cast<R *>(smem);
    R *sy = sx + a.nmax;
    R *sz = sy + a.nmax;
    uint8_t *spc = reinterpret_cast<uint8_t *>(sz + a.nmax);
    __shared__ int s_next;
    __shared__ R s_sigma[TTS_MAX_SPECIES][2];
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
        // the bath of every step was computed before this launch
        const R *sig_traj = a.traj_sig + int64_t(I.inst) * a.traj_cap * 4;
        const double *T_traj = a.traj_T + int64_t(I.inst) * a.traj_cap * 2;
        __syncthreads();
        // merged sweep: colour 0 left half a step ahead by the previous step
        const bool mer = a.merged && I.ncolours >= 2;
        bool open = mer && !a.first_chunk && a.open_state[I.inst] != 0;
        for (int64_t st = 0; st < nsteps; ++st) {
            const int64_t step = step0 + st;
            if (threadIdx.x < 4) (&s_sigma[0][0])[threadIdx.x] = sig_traj[st * 4 + threadIdx.x];
            __syncthreads();
            const int K = I.ncolours;
            const bool close = !mer || (a.last_chunk && st == nsteps - 1) ||
                               (a.sample_every > 0 && (step + 1) % a.sample_every == 0);
            for (int p = 0; p < 2 * K - 1; ++p) {
                if (mer && p == 2 * K - 2 && !close) continue;     // the trailing half waits for the bridge
                const int c = p < K - 1 ? p : (p == K - 1 ? K - 1 : 2 * K - 2 - p);
                const int hsel = (p == K - 1 || (mer && p == 0 && open)) ? 1 : 0;
                const R h = hsel ? R(a.dt) : R(0.5 * a.dt);
                const int beg = I.colour_begin[c], end = I.colour_begin[c + 1];
                if constexpr (sizeof(R) == 4) {
                    resident_pair_pass<AXZ>(a, I, sx, sy, sz, spc, beg, end, step, p, hsel, s_sigma);
                } else {
                    for (int idx = beg + threadIdx.x; idx < end; idx += blockDim.x) {
                        const uint32_t at = static_cast<uint32_t>(a.atom[I.slot_begin + idx]);
                        R htx, hty, htz, h1x, h1y, h1z;
                        resident_sums<R>(at, I, sx, sy, sz, spc, htx, hty, htz, h1x, h1y, h1z);
                        const int t = spc[at];
                        const FastSpecies<R> sp = t ? a.sp[1] : a.sp[0];
                        R s0 = sx[at], s1 = sy[at], s2 = sz[at];
                        const R sig = s_sigma[t][hsel];
                        if (sig > R(0)) {
                            const u32x4 w = philox4x32_10(
                                u32x4{at, static_cast<uint32_t>(step), static_cast<uint32_t>(p), I.inst_global}, a.key0,
                                a.key1);
                            fast_update<R, AXZ>(s0, s1, s2, htx, hty, htz, h1x, h1y, h1z, sp, R(a.axis[0]),
                                                R(a.axis[1]), R(a.axis[2]), R(a.B[0]), R(a.B[1]), R(a.B[2]), sig, &w, h);
                        } else {
                            fast_update<R, AXZ>(s0, s1, s2, htx, hty, htz, h1x, h1y, h1z, sp, R(a.axis[0]),
                                                R(a.axis[1]), R(a.axis[2]), R(a.B[0]), R(a.B[1]), R(a.B[2]), sig,
                                                nullptr, h);
                        }
                        sx[at] = s0;
                        sy[at] = s1;
                        sz[at] = s2;
                    }
                }
                __syncthreads();
            }
            open = mer && !close;
            if (a.sample_every > 0 && (step + 1) % a.sample_every == 0)
                resident_observe<R>(a, I, sx, sy, sz, spc, step + 1, T_traj[2 * st], T_traj[2 * st + 1], warp_red);
        }
        if (threadIdx.x == 0) a.open_state[I.inst] = open ? 1 : 0;
        for (int s = threadIdx.x; s < I.n; s += blockDim.x) {
            const int64_t slot = I.slot_begin + s;
            const int at = a.atom[slot];
            const R v0 = sx[at], v1 = sy[at], v2 = sz[at];
            if (!(isfinite(v0) && isfinite(v1) && isfinite(v2))) atomicOr(a.health, kHealthNonFinite);
            a.sx[slot] = v0;
            a.sy[slot] = v1;
            a.sz[slot] = v2;
        }
        __syncthreads();
    }
}

// One thread per instance: the one-cell bath of `nsteps` steps from the
// current step -- the noise table of each step from T_e(t_n), then the
// two-temperature advance t_n -> t_n+1 -- independent of the spins (the spins
// do not heat the electrons), so every instance's trajectory is computed
// before the spin kernel runs instead of serially inside it.
template <typename R>
__global__ void resident_traj_kernel(ResArgs<R> a, int nsteps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_inst) return;
    const DevInstance D = a.inst[i];
    const int64_t step0 = *a.step;
    double T[2] = {a.Te[D.cell_begin], a.Tl[D.cell_begin]};
    double deposited = 0.0;
    R *sig = a.traj_sig + int64_t(i) * a.traj_cap * 4;
    double *TT = a.traj_T + int64_t(i) * a.traj_cap * 2;
    for (int st = 0; st < nsteps; ++st) {
        resident_bath<R>(a, D, step0 + st, 0, T, &deposited, sig + 4 * st);
        if (a.ttm_active) resident_bath<R>(a, D, step0 + st, 1, T, &deposited, nullptr);
        TT[2 * st] = T[0];
        TT[2 * st + 1] = T[1];
    }
    a.Te[D.cell_begin] = T[0];
    a.Tl[D.cell_begin] = T[1];
    if (a.ttm_active) a.src_energy[i] += deposited;
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
    void *S1 = nullptr;              // FP32: second state buffer (= S unless the fused sweep is offered)
    int *cur = nullptr;              // FP32: which of S / S1 holds the current state
    unsigned *done = nullptr;        // fused sweep: CTAs finished in the running launch
    SweepShape sweep{};              // fused sweep launch shape (sweep.C == 0: not offered)
    CheckerInst *ci = nullptr;
    int64_t work = 0;
    int K = 2;
    uint32_t shape[3] = {0, 0, 0};   // cells of every instance
    uint32_t inst_base = 0;
    int bx = 64, by = 4;             // pass block shape
    bool axis_z = false;             // anisotropy axis is +z
    bool pair = false;               // FP32 checker on site pairs
    bool noise = false;              // some species has alpha > 0
    TileArgs tile{};                 // pair engine staged in shared memory (bx = by = 0)
    int cell_formula = 0;            // the pair kernels compute the TTM cell of a site
    int cell0 = 0, cstride = 0;
    uint32_t ncell[3] = {1, 1, 1};
    size_t tile_smem = 0;
    int tile_grid = 0;
    // checker: (bx, by, instance chains); resident: (threads, 0, 1)
    struct Cfg {
        int first, second;
        int chains = 1;
    };
    std::vector<Cfg> configs;
    int config = 0;
    // FP32 separate passes: instances split into `chains` groups whose passes
    // run on parallel streams (graph branches), so that one group's pass
    // boundary overlaps another group's pass
    int chains = 1;
    static constexpr int kMaxChains = 4;
    cudaStream_t side[kMaxChains] = {};      // chains 2.. and the TTM branch
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxChains - 1] = {};
    cudaEvent_t ev_ttm = nullptr;    // the step's TTM, run beside the chains
    // resident
    ResInst *ri = nullptr;
    int *order = nullptr;
    int *queue = nullptr;
    void *traj_sig = nullptr;        // resident: bath trajectory of a chunk of steps
    double *traj_T = nullptr;
    int *open_state = nullptr;
    int traj_cap = 256;
    int nmax = 0;
    int sm_count = 0;
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

f2 host_f2(double a, double b)
{
    const float fa = static_cast<float>(a), fb = static_cast<float>(b);
    uint32_t ua, ub;
    std::memcpy(&ua, &fa, 4);
    std::memcpy(&ub, &fb, 4);
    return f2{static_cast<unsigned long long>(ua) | (static_cast<unsigned long long>(ub) << 32)};
}
f2 host_splat(double a) { return host_f2(a, a); }

// Constants of one pass of the pair kernel (h = dt / 2 or dt).
PairConsts make_pair_consts(const EngineState *e, const StepParams &p, int hsel)
{
    const double h = hsel ? p.dt : 0.5 * p.dt;
    const FastSpecies<double> *sp = e->spd;
    auto cd = [](double v0, double v1, f2 &c, f2 &d) {
        c = host_splat(v0);
        d = host_splat(v1 - v0);
    };
    PairConsts k{};
    cd(sp[0].J0, sp[1].J0, k.J0c, k.J0d);
    cd(sp[0].J1 - sp[0].J0, sp[1].J1 - sp[1].J0, k.dJc, k.dJd);
    cd(sp[0].kappa, sp[1].kappa, k.kc, k.kd);
    cd(sp[0].alpha, sp[1].alpha, k.alc, k.ald);
    cd(-0.5 * sp[0].kappa * sp[0].gprime * h, -0.5 * sp[1].kappa * sp[1].gprime * h, k.khgc, k.khgd);
    cd(sp[0].gprime * h, sp[1].gprime * h, k.ghc, k.ghd);
    const double log2e = 1.0 / std::log(2.0);
    cd(-sp[0].alpha * log2e, -sp[1].alpha * log2e, k.nalc, k.nald);
    k.nx = host_splat(p.axis[0]);
    k.ny = host_splat(p.axis[1]);
    k.nz = host_splat(p.axis[2]);
    k.Bx = host_splat(p.B[0]);
    k.By = host_splat(p.B[1]);
    k.Bz = host_splat(p.B[2]);
    k.one = host_splat(1.0);
    k.neg1 = host_splat(-1.0);
    k.u_off = host_splat(std::ldexp(1.0, -24) - 1.0);
    k.m2ln2 = host_splat(-2.0 * std::log(2.0));
    k.twopi = host_splat(2.0 * M_PI);
    k.negpi = host_splat(-M_PI);
    k.s3 = host_splat(-1.0 / 6.0);
    k.s5 = host_splat(1.0 / 120.0);
    k.c2 = host_splat(-0.5);
    k.c4 = host_splat(1.0 / 24.0);
    k.c6 = host_splat(-1.0 / 720.0);
    return k;
}

size_t resident_bytes(int n, int precision) { return size_t(n) * (3 * (precision == 64 ? 8 : 4) + 1) + 16; }

const void *resident_fn(int precision, bool axis_z)
{
    if (precision == 64)
        return axis_z ? reinterpret_cast<const void *>(resident_kernel<double, true>)
                      : reinterpret_cast<const void *>(resident_kernel<double, false>);
    return axis_z ? reinterpret_cast<const void *>(resident_kernel<float, true>)
                  : reinterpret_cast<const void *>(resident_kernel<float, false>);
}

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
    // grid (x blocks, Lz, instances): y and z are limited to 65535
    even_equal = even_equal && host[0].cells[2] <= 65535 && host.size() <= 65535;
    if (requested == TTS_ENGINE_RESIDENT) return fits ? TTS_ENGINE_RESIDENT : -1;
    if (requested == TTS_ENGINE_CHECKER) return even_equal ? TTS_ENGINE_CHECKER : -1;
    // AUTO: many small instances -> resident; otherwise large even lattices -> checker
    if (fits && host.size() >= 8) return TTS_ENGINE_RESIDENT;
    if (even_equal) return TTS_ENGINE_CHECKER;
    if (fits) return TTS_ENGINE_RESIDENT;
    return -1;
}

namespace {
// Does cell0 + i cstride + (cz ncy + cy) ncx + cx, c_k = floor(k n_k / L_k),
// reproduce the cell map of every checker slot?  Sets the engine's formula.
void check_cell_formula(EngineState *e, const std::vector<DevInstance> &dinst, const std::vector<int> &cellmap)
{
    e->cell_formula = 0;
    if (!e->pair || dinst.empty() || int64_t(cellmap.size()) != e->n_total) return;
    const DevInstance &d0 = dinst[0];
    const int cstride = dinst.size() > 1 ? dinst[1].cell_begin - d0.cell_begin : d0.ncells;
    uint32_t nc[3];
    for (int k = 0; k < 3; ++k) nc[k] = static_cast<uint32_t>(std::max(1, d0.cells[k]));
    if (int64_t(nc[0]) * nc[1] * nc[2] != d0.ncells && !(d0.ncells == 1)) return;
    if (d0.ncells == 1) nc[0] = nc[1] = nc[2] = 1;
    for (size_t i = 0; i < dinst.size(); ++i)
        if (dinst[i].cell_begin != d0.cell_begin + int(i) * cstride || dinst[i].ncells != d0.ncells ||
            dinst[i].slot_begin != int64_t(i) * (e->n_total / e->n_inst))
            return;
    const uint32_t Lx = e->shape[0], Ly = e->shape[1], Lz = e->shape[2], hx = Lx / 2;
    const uint32_t L[3] = {Lx, Ly, Lz};
    for (int k = 0; k < 3; ++k)
        if (!fastdiv_ok(L[k], L[k] * nc[k])) return;
    const int64_t per = e->n_total / e->n_inst, nhalf = per / 2;
    for (size_t i = 0; i < dinst.size(); ++i)
        for (int64_t s = 0; s < per; ++s) {
            const int64_t colour = s / nhalf, r = s - colour * nhalf;
            const uint32_t z = static_cast<uint32_t>(r / (int64_t(Ly) * hx));
            const uint32_t y = static_cast<uint32_t>((r / hx) % Ly), kx = static_cast<uint32_t>(r % hx);
            const uint32_t x = 2 * kx + ((y + z + uint32_t(colour)) & 1u);
            const uint32_t cx = x * nc[0] / Lx, cy = y * nc[1] / Ly, cz = z * nc[2] / Lz;
            const int want = d0.cell_begin + int(i) * cstride + int((cz * nc[1] + cy) * nc[0] + cx);
            if (cellmap[size_t(int64_t(i) * per + s)] != want) return;
        }
    e->cell0 = d0.cell_begin;
    e->cstride = cstride;
    for (int k = 0; k < 3; ++k) e->ncell[k] = nc[k];
    e->cell_formula = 1;
}

// Shape check and launch set-up of the shared-memory staged pair pass: hx a
// power of two in [8, 256], tile rows by = the largest divisor of Ly/2 with
// by hx <= 256, one wave of CTAs over the (column, z) planes.
bool setup_tiled(EngineState *e)
{
    const uint32_t hx = e->shape[0] / 2, Ly2 = e->shape[1] / 2, Lz = e->shape[2];
    if (hx < 8 || hx > 256 || (hx & (hx - 1)) != 0 || Ly2 < 1) return false;
    uint32_t by = 0;
    for (uint32_t c = std::min<uint32_t>(256 / hx, Ly2); c >= 1; --c)
        if (Ly2 % c == 0) {
            by = c;
            break;
        }
    if (by == 0) return false;
    TileArgs t{};
    t.by = by;
    t.hx_shift = 0;
    while ((1u << t.hx_shift) < hx) ++t.hx_shift;
    t.nyb = Ly2 / by;
    t.ncol = static_cast<uint32_t>(e->n_inst) * t.nyb;
    t.units = uint64_t(t.ncol) * Lz;
    const size_t to = size_t(by + 2) * hx, tw = size_t(by) * hx;
    const size_t smem = (8 * to + 4 * tw) * 16 + 6 * sizeof(uint64_t);
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (const void *fn : {reinterpret_cast<const void *>(checker_pair_tiled_kernel<true, false>),
                           reinterpret_cast<const void *>(checker_pair_tiled_kernel<false, false>),
                           reinterpret_cast<const void *>(checker_pair_tiled_kernel<true, true>),
                           reinterpret_cast<const void *>(checker_pair_tiled_kernel<false, true>)}) {
        int ps = 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, fn, 256, smem) != cudaSuccess || ps < 1) {
            cudaGetLastError();
            return false;
        }
        per_sm = per_sm == 0 ? ps : std::min(per_sm, ps);
    }
    e->tile = t;
    e->tile_smem = smem;
    e->tile_grid = static_cast<int>(std::min<uint64_t>(t.units, uint64_t(nsm) * per_sm));
    return true;
}
}  // namespace

// Launch shape of the fused sweep: R = the largest divisor of Ly/2 with
// R hx <= 256 pair columns (3 R hx threads), clusters of C = Ly/2 / R <= 16
// CTAs, shared memory for the plane rings, and the number of z segments per
// instance that minimises (waves of clusters) x (planes per segment + 6).
bool setup_sweep(EngineState *e)
{
    const uint32_t hx = e->shape[0] / 2, Ly2 = e->shape[1] / 2, Lz = e->shape[2];
    if (e->K != 2 || hx < 1 || Ly2 < 1 || Lz < 4) return false;
    uint32_t R = 0;
    for (uint32_t c = std::min<uint32_t>(256 / hx, Ly2); c >= 1; --c)
        if (Ly2 % c == 0) {
            R = c;
            break;
        }
    if (R == 0) return false;
    const uint32_t C = Ly2 / R;
    if (C > 16) return false;
    SweepShape sh;
    sh.R = R;
    sh.C = C;
    sh.threads = 3 * R * hx;
    sh.smem = sweep_smem_bytes(R * hx, hx);
    if (sh.smem > 227u * 1024u) return false;
    int nclusters = 0;
    for (const void *fn : {reinterpret_cast<const void *>(checker_sweep_kernel<true>),
                           reinterpret_cast<const void *>(checker_sweep_kernel<false>)}) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sh.smem)) !=
                cudaSuccess ||
            (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
            cudaGetLastError();
            return false;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(sh.threads, 1, 1);
        cfg.dynamicSmemBytes = sh.smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0, per_sm = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess || n < 1 ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, static_cast<int>(sh.threads), sh.smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            return false;
        }
        // clusters resident at once: never more than the SMs hold CTAs
        if (e->sm_count > 0) n = std::min(n, e->sm_count * per_sm / static_cast<int>(C));
        if (n < 1) return false;
        nclusters = nclusters == 0 ? n : std::min(nclusters, n);
    }
    double best = 0.0;
    for (uint32_t s = 1; s <= std::max<uint32_t>(1, Lz / 4); ++s) {
        const uint64_t clusters = uint64_t(s) * e->n_inst;
        const double waves = double((clusters + nclusters - 1) / nclusters);
        const double cost = waves * (double((Lz + s - 1) / s) + 6.0);
        if (best == 0.0 || cost < best) {
            best = cost;
            sh.nseg = s;
        }
    }
    e->sweep = sh;
    return true;
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
    for (int t = 0; t < d.nspecies; ++t) e->noise = e->noise || d.alpha[t] > 0.0;
    {
        const double an = std::sqrt(d.axis[0] * d.axis[0] + d.axis[1] * d.axis[1] + d.axis[2] * d.axis[2]);
        e->axis_z = an > 0.0 && d.axis[0] == 0.0 && d.axis[1] == 0.0 && d.axis[2] > 0.0;
    }
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
        for (int k = 0; k < 3; ++k) e->shape[k] = static_cast<uint32_t>(host[0].cells[k]);
        e->inst_base = static_cast<uint32_t>(d.instance_base);
        e->pair = d.precision == 32;
        {
            int dev = 0, nsm = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
                e->sm_count = nsm;
            else
                cudaGetLastError();
        }
        // x rows of hx = Lx/2 colour sites in warps, the rest of the threads in y
        const int hxs = static_cast<int>(e->shape[0] / 2);
        if (e->pair) {
            // (bx, by) pairs x pair rows; (0, 0): the shared-memory staged
            // pass.  Default: 128 threads.
            e->bx = hxs >= 64 ? 64 : 32;
            e->by = 128 / e->bx;
            for (int bx : {32, 64, 128})
                if (bx <= std::max(32, hxs))
                    for (int threads : {128, 256}) e->configs.push_back({bx, threads / bx});
        } else {
            // FP64: a row of at most hx sites a block row, and blocks small
            // enough that every SM gets one (a pass's FP64 work runs at the
            // FP64 rate of the SMs it lands on: on 32^3, 256-thread blocks
            // filled 128 SMs half-idle).
            int bx = 128;
            while (bx > 8 && bx > hxs) bx >>= 1;
            const int nsm = e->sm_count > 0 ? e->sm_count : 148;
            auto nblocks = [&](int threads) {
                const int64_t rows = (e->shape[1] + threads / bx - 1) / (threads / bx);
                return int64_t((hxs + bx - 1) / bx) * rows * e->shape[2] * e->n_inst;
            };
            int threads = 256;
            while (threads > std::max(32, bx) && nblocks(threads) < nsm) threads >>= 1;
            e->bx = bx;
            e->by = threads / bx;
            e->configs.push_back({e->bx, e->by});
            for (int cbx : {32, 64, 128})
                if (cbx <= std::max(32, hxs))
                    for (int t : {128, 256})
                        if (t / cbx >= 1 && !(cbx == e->bx && t / cbx == e->by)) e->configs.push_back({cbx, t / cbx});
        }
        // the default first
        for (size_t k = 0; k < e->configs.size(); ++k)
            if (e->configs[k].first == e->bx && e->configs[k].second == e->by) {
                std::swap(e->configs[0], e->configs[k]);
                break;
            }
        e->config = 0;
        if (e->pair) {
            std::vector<int> cm(static_cast<size_t>(e->n_total));
            if (cudaStreamSynchronize(st) == cudaSuccess &&
                cudaMemcpy(cm.data(), b.cell, cm.size() * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
                check_cell_formula(e, dinst, cm);
            else
                cudaGetLastError();
            if (setup_tiled(e)) e->configs.push_back({0, 0});
            // The default block shape with the instances in 2 or 4 chains:
            // on GdFeCo 128^3 x 4 two chains took a step from 146 to 142 us
            // (the colour passes alone 150 -> 139 us), four 143 us.  With two
            // or more instances two chains become the default.
            if (e->n_inst >= 2) {
                bool ok = cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventCreateWithFlags(&e->ev_ttm, cudaEventDisableTiming) == cudaSuccess;
                for (int c = 0; ok && c < EngineState::kMaxChains; ++c)
                    ok = cudaStreamCreateWithFlags(&e->side[c], cudaStreamNonBlocking) == cudaSuccess &&
                         (c == EngineState::kMaxChains - 1 ||
                          cudaEventCreateWithFlags(&e->ev_join[c], cudaEventDisableTiming) == cudaSuccess);
                if (ok) {
                    const EngineState::Cfg d = e->configs[0];
                    e->configs.insert(e->configs.begin(), {d.first, d.second, 2});
                    if (e->n_inst >= 4) e->configs.push_back({d.first, d.second, 4});
                    e->chains = 2;
                } else {
                    cudaGetLastError();
                }
            }
        }
        const size_t vs = d.precision == 64 ? sizeof(double4a) : sizeof(float4);
        const bool sweep = e->pair && setup_sweep(e);
        if ((ce = cudaMalloc(&e->S, size_t(e->n_total) * vs)) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->ci), ci.size() * sizeof(CheckerInst))) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->cur), sizeof(int))) != cudaSuccess ||
            (sweep && (ce = cudaMalloc(&e->S1, size_t(e->n_total) * vs)) != cudaSuccess) ||
            (sweep && (ce = cudaMalloc(reinterpret_cast<void **>(&e->done), sizeof(unsigned))) != cudaSuccess)) {
            cudaGetLastError();
            engine_destroy(e);
            return eng_fail(TTS_ERR_OOM, std::string("checker buffers: ") + cudaGetErrorString(ce));
        }
        cudaMemsetAsync(e->cur, 0, sizeof(int), st);
        if (sweep) {
            cudaMemsetAsync(e->done, 0, sizeof(unsigned), st);
            // offered to the autotuner; the separate passes stay the default
            // (on 128^3 x 4 they measured about twice as fast: the fused
            // launch is bound by the latency of one update a warp per step).
            // Fusion depth: z segments per instance 1, 2, 4, 8 (each at least
            // four planes long), then the cost model's choice, last.
            for (uint32_t sg : {1u, 2u, 4u, 8u})
                if (sg != e->sweep.nseg && sg <= e->shape[2] / 4) e->configs.push_back({-2, static_cast<int>(sg)});
            e->configs.push_back({-2, 0});
        } else {
            e->S1 = e->S;
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
        const void *fn = resident_fn(d.precision, e->axis_z);
        cudaError_t a1 = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(e->smem));
        int per_sm = 0;
        if (a1 == cudaSuccess) a1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, e->block, e->smem);
        if (a1 != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            delete e;
            return eng_fail(TTS_ERR_UNSUPPORTED, "resident kernel does not fit one CTA per SM");
        }
        e->grid = std::min(e->n_inst, nsm * per_sm);
        e->configs.push_back({512, 0});
        for (int threads : {256, 384}) {
            int ps = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, fn, threads, e->smem) == cudaSuccess && ps >= 1)
                e->configs.push_back({threads, 0});
            cudaGetLastError();
        }
        e->sm_count = nsm;
        if ((ce = cudaMalloc(reinterpret_cast<void **>(&e->ri), ri.size() * sizeof(ResInst))) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->order), order.size() * sizeof(int))) != cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->queue), sizeof(int))) != cudaSuccess ||
            (ce = cudaMalloc(&e->traj_sig, size_t(e->n_inst) * e->traj_cap * 4 * (d.precision == 64 ? 8 : 4))) !=
                cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->traj_T), size_t(e->n_inst) * e->traj_cap * 2 * sizeof(double))) !=
                cudaSuccess ||
            (ce = cudaMalloc(reinterpret_cast<void **>(&e->open_state), size_t(e->n_inst) * sizeof(int))) != cudaSuccess) {
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
    for (int c = 0; c < EngineState::kMaxChains; ++c)
        if (e->side[c]) cudaStreamDestroy(e->side[c]);
    for (int c = 0; c < EngineState::kMaxChains - 1; ++c)
        if (e->ev_join[c]) cudaEventDestroy(e->ev_join[c]);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    if (e->ev_ttm) cudaEventDestroy(e->ev_ttm);
    if (e->S1 && e->S1 != e->S) cudaFree(e->S1);
    for (void *q : {static_cast<void *>(e->cur), static_cast<void *>(e->done)})
        if (q) cudaFree(q);
    for (void *q : {e->S, static_cast<void *>(e->ci), static_cast<void *>(e->ri), static_cast<void *>(e->order),
                    static_cast<void *>(e->queue), e->traj_sig, static_cast<void *>(e->traj_T),
                    static_cast<void *>(e->open_state)})
        if (q) cudaFree(q);
    delete e;
}

bool engine_multi_step(const EngineState *e) { return e && e->engine == TTS_ENGINE_RESIDENT; }

int engine_num_configs(const EngineState *e) { return e ? static_cast<int>(e->configs.size()) : 0; }
int engine_config(const EngineState *e) { return e ? e->config : 0; }

void engine_set_config(EngineState *e, int index)
{
    if (!e || index < 0 || index >= static_cast<int>(e->configs.size())) return;
    e->config = index;
    if (e->engine == TTS_ENGINE_CHECKER) {
        e->bx = e->configs[index].first;
        e->by = e->configs[index].second;
        e->chains = e->configs[index].chains;
    } else if (e->engine == TTS_ENGINE_RESIDENT) {
        e->block = e->configs[index].first;
        int ps = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, resident_fn(e->precision, e->axis_z), e->block, e->smem) !=
                cudaSuccess ||
            ps < 1) {
            cudaGetLastError();
            ps = 1;
        }
        e->grid = std::min(e->n_inst, e->sm_count * ps);
    }
}

namespace {
// Block shape (pairs or sites along x, rows) of the separate-pass kernels;
// with the fused sweep selected (bx < 0) the merged sweep's passes run
// checker_pair_kernel on its default shape.
void row_block(const EngineState *e, int &bx, int &by)
{
    bx = e->bx;
    by = e->by;
    if (bx < 0) {
        bx = e->shape[0] / 2 >= 64 ? 64 : 32;
        by = 128 / bx;
    }
}

// The cell mode of the pair kernels for these arguments.
int pair_cell_mode(const PairArgs &a)
{
    if (!a.cell_formula) return kCellMap;
    return a.shx >= 0 && a.shy >= 0 && a.shz >= 0 ? kCellShift : kCellDiv;
}

using PairKernelFn = void (*)(PairArgs, int, int, int);

template <bool AXZ, bool SW>
PairKernelFn pair_kernel_fn_cm(int cm)
{
    return cm == kCellShift ? checker_pair_kernel<AXZ, SW, kCellShift>
                            : (cm == kCellDiv ? checker_pair_kernel<AXZ, SW, kCellDiv> : checker_pair_kernel<AXZ, SW, kCellMap>);
}

PairKernelFn pair_kernel_fn(bool axz, bool sw, int cm)
{
    return axz ? (sw ? pair_kernel_fn_cm<true, true>(cm) : pair_kernel_fn_cm<true, false>(cm))
               : (sw ? pair_kernel_fn_cm<false, true>(cm) : pair_kernel_fn_cm<false, false>(cm));
}

// Launch arguments of the FP32 pair kernels for a pass with step h(hsel).
PairArgs pair_args(const EngineState *e, const StepParams &p, const DevBuffers &b, int hsel)
{
    PairArgs a{};
    a.S = static_cast<ulonglong2 *>(e->S);
    a.S1 = static_cast<ulonglong2 *>(e->S1);
    a.cur = e->cur;
    a.cell = b.cell;
    // with sigma_alternate the table of odd steps is sigma_alt; the parity of
    // the step is fixed when the step is recorded
    a.sigma = static_cast<const float *>(p.sigma_alternate && p.sigma_parity ? b.sigma_alt : b.sigma);
    a.step = b.step;
    a.health = b.health;
    a.k = make_pair_consts(e, p, hsel);
    a.rk = philox_round_keys(p.key0, p.key1);
    a.Lx = e->shape[0];
    a.Ly = e->shape[1];
    a.Lz = e->shape[2];
    a.hx = e->shape[0] / 2;
    a.Ly2 = e->shape[1] / 2;
    {
        int bx, by;
        row_block(e, bx, by);
        a.nkx = bx ? (a.hx + bx - 1) / bx : 0;
        a.dnkx = make_fastdiv(std::max<uint32_t>(a.nkx, 1));
    }
    a.nhalf = static_cast<uint32_t>(e->n_total / e->n_inst / 2);
    a.npair = a.nhalf / 2;
    a.n_inst_sites = e->n_total / e->n_inst;
    a.inst_base = e->inst_base;
    a.noise = e->noise ? 1 : 0;
    a.n_inst = e->n_inst;
    a.cell_formula = e->cell_formula;
    a.cell0 = e->cell0;
    a.cstride = e->cstride;
    a.ncx = e->ncell[0];
    a.ncy = e->ncell[1];
    a.ncz = e->ncell[2];
    a.dLx = make_fastdiv(e->shape[0]);
    a.dLy = make_fastdiv(e->shape[1]);
    a.dLz = make_fastdiv(e->shape[2]);
    // two planes ahead: measured 5 % faster than none on the 128^3 x 4 benchmark
    // (one to four planes all gave the same; a wave of blocks ahead, 37 planes, 0.6 %)
    a.pf_planes = 2;
    int *sh[3] = {&a.shx, &a.shy, &a.shz};
    for (int k = 0; k < 3; ++k) {
        *sh[k] = -1;
        const uint32_t L = e->shape[k], n = e->ncell[k];
        if (n > 0 && L % n == 0) {
            const uint32_t q = L / n;
            if ((q & (q - 1)) == 0) {
                int b = 0;
                while ((1u << b) < q) ++b;
                *sh[k] = b;
            }
        }
    }
    return a;
}

void launch_pair_to_general(EngineState *e, const DevBuffers &b, cudaStream_t st, int sample_every, int conditional)
{
    const int bs = 256;
    const int64_t np = e->n_total / 2;
    pair_to_general_kernel<<<(np + bs - 1) / bs, bs, 0, st>>>(
        static_cast<const float4 *>(e->S), static_cast<const float4 *>(e->S1), e->cur, static_cast<float *>(b.sx),
        static_cast<float *>(b.sy),
        static_cast<float *>(b.sz), np, e->shape[0] / 2, e->shape[1] / 2,
        static_cast<uint32_t>(e->n_total / e->n_inst / 4), b.step, sample_every, conditional);
}
}  // namespace

cudaError_t engine_obs_partials(EngineState *e, const StepParams &p, const DevBuffers &b, int mode, cudaStream_t st)
{
    if (!e || e->engine != TTS_ENGINE_CHECKER || !e->pair) return cudaErrorNotSupported;
    PairObsArgs o{};
    o.obs_block_inst = b.obs_block_inst;
    o.inst = b.inst;
    o.obs_partial = b.obs_partial;
    o.obs_blocks = p.obs_blocks;
    o.sample_every = p.sample_every;
    for (int t = 0; t < TTS_MAX_SPECIES; ++t) {
        o.mu[t] = p.sp[t].mu;
        o.K[t] = p.sp[t].K;
    }
    const int grid = p.obs_blocks < 1184 ? p.obs_blocks : 1184;
    checker_pair_obs_kernel<<<grid, kObsBlock, 0, st>>>(pair_args(e, p, b, 0), o, mode);
    return cudaGetLastError();
}

bool engine_step_parity(const EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                        bool ttm_active)
{
    const bool chains = e->engine == TTS_ENGINE_CHECKER && e->pair && !p.merged && e->bx > 0 &&
                        std::min(e->chains, e->n_inst) > 1;
    return chains && ttm_active && p.ttm_one_substep && !p.sigma_per_step && tp.source != TTS_SOURCE_STEP_PROFILE &&
           b.sigma_alt && b.cell_inst;
}

cudaError_t engine_record_step(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                               bool ttm_active, cudaStream_t st, int *kernels, cudaEvent_t ev0, cudaEvent_t ev1)
{
    *kernels = 0;
    if (e->engine != TTS_ENGINE_CHECKER) return cudaErrorNotSupported;
    cudaError_t err = cudaSuccess;
    if (p.sigma_per_step) {
        err = launch_sigma(p, b, p.ncells_total, e->precision, st);
        ++*kernels;
    }
    if (err == cudaSuccess && ev0) err = cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal);
    const int npass = 2 * e->K - 1;
    // merged sweep: the first pass leads (dt/2 or a dt bridge), the last trails
    auto ctl = [&](int pass) {
        SweepCtl w;
        if (!p.merged) return w;
        w.mode = pass == 0 ? 1 : (pass == npass - 1 ? 2 : 0);
        w.open = b.open;
        w.target = b.target;
        w.sample_every = p.sample_every;
        return w;
    };
    const bool fused = e->pair && e->bx == -2 && !p.merged;
    if (fused && err == cudaSuccess) {
        // the three passes of the step in one launch (checker_sweep_kernel)
        PairArgs a = pair_args(e, p, b, 0);
        SweepArgs w{};
        const uint32_t nseg = e->by > 0 ? static_cast<uint32_t>(e->by) : e->sweep.nseg;
        w.R = e->sweep.R;
        w.nseg = nseg;
        w.done = e->done;
        w.ctas = e->sweep.C * nseg * static_cast<uint32_t>(e->n_inst);
        w.cur = e->cur;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(e->sweep.C, nseg, e->n_inst);
        cfg.blockDim = dim3(e->sweep.threads, 1, 1);
        cfg.dynamicSmemBytes = e->sweep.smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = e->sweep.C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        err = e->axis_z ? cudaLaunchKernelEx(&cfg, checker_sweep_kernel<true>, a, w)
                        : cudaLaunchKernelEx(&cfg, checker_sweep_kernel<false>, a, w);
        ++*kernels;
    }
    // instance chains of the FP32 separate passes (not for the merged sweep)
    const int chains = (e->pair && !fused && !p.merged && e->bx > 0) ? std::min(e->chains, e->n_inst) : 1;
    // With chains, a one-sub-step TTM runs on a branch of its own beside the
    // colour passes (it does not depend on the spins): it writes the next
    // step's noise table into the table of that step's parity while the
    // passes read the other, and the step counter advances after the passes.
    // (Not while profiling: the colour passes are then timed on their own.)
    const bool ttm_beside = engine_step_parity(e, p, b, tp, ttm_active) && !ev0;
    StepParams q = p;
    q.sigma_alternate = ttm_beside ? 1 : 0;
    if (chains > 1 && err == cudaSuccess) {
        err = cudaEventRecord(e->ev_fork, st);
        for (int c = 1; c < chains && err == cudaSuccess; ++c) err = cudaStreamWaitEvent(e->side[c - 1], e->ev_fork, 0);
        cudaStream_t tst = e->side[chains - 1];
        if (ttm_beside && err == cudaSuccess) {
            err = cudaStreamWaitEvent(tst, e->ev_fork, 0);
            if (err == cudaSuccess) err = launch_ttm(q, b, tp, p.n_instances, tst, e->precision, 0);
            if (err == cudaSuccess) err = cudaEventRecord(e->ev_ttm, tst);
            *kernels += 2;
        }
        for (int pass = 0; pass < npass && err == cudaSuccess; ++pass) {
            const int c = pass < e->K - 1 ? pass : (pass == e->K - 1 ? e->K - 1 : 2 * e->K - 2 - pass);
            const int hsel = pass == e->K - 1 ? 1 : 0;
            int rbx, rby;
            row_block(e, rbx, rby);
            PairArgs a = pair_args(e, q, b, hsel);
            const auto fn = pair_kernel_fn(e->axis_z, false, pair_cell_mode(a));
            for (int ch = 0; ch < chains && err == cudaSuccess; ++ch) {
                const int i0 = ch * e->n_inst / chains, i1 = (ch + 1) * e->n_inst / chains;
                a.inst0 = i0;
                const dim3 pgrid(a.nkx * ((a.Ly2 + rby - 1) / rby), e->shape[2], i1 - i0);
                fn<<<pgrid, dim3(rbx, rby), 0, ch ? e->side[ch - 1] : st>>>(a, c, hsel, pass);
                err = cudaGetLastError();
                ++*kernels;
            }
        }
        for (int c = 1; c < chains && err == cudaSuccess; ++c) {
            err = cudaEventRecord(e->ev_join[c - 1], e->side[c - 1]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(st, e->ev_join[c - 1], 0);
        }
    }
    for (int pass = 0; pass < npass && err == cudaSuccess && !fused && chains == 1; ++pass) {
        const int c = pass < e->K - 1 ? pass : (pass == e->K - 1 ? e->K - 1 : 2 * e->K - 2 - pass);
        const int hsel = pass == e->K - 1 ? 1 : 0;
        int rbx, rby;
        row_block(e, rbx, rby);
        const dim3 block(rbx, rby);
        const uint32_t nkx = rbx ? (e->shape[0] / 2 + rbx - 1) / rbx : 0;
        const dim3 grid(rby ? nkx * ((e->shape[1] + rby - 1) / rby) : 0, e->shape[2], e->n_inst);
        auto fill_shape = [&](auto &a) {
            a.nkx = nkx;
            a.Lx = e->shape[0];
            a.Ly = e->shape[1];
            a.Lz = e->shape[2];
            a.hx = e->shape[0] / 2;
            a.nhalf = static_cast<uint32_t>(e->n_total / e->n_inst / 2);
            a.n_inst_sites = e->n_total / e->n_inst;
            a.inst_base = e->inst_base;
        };
        if (e->precision == 64) {
            CheckerArgs<double> a{};
            a.S = static_cast<double4a *>(e->S);
            fill_shape(a);
            a.sw = ctl(pass);
            a.cell = b.cell;
            a.sigma = static_cast<const double *>(b.sigma);
            a.step = b.step;
            a.health = b.health;
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spd[t];
            a.nx = p.axis[0]; a.ny = p.axis[1]; a.nz = p.axis[2];
            a.Bx = p.B[0]; a.By = p.B[1]; a.Bz = p.B[2];
            a.dt = p.dt;
            a.key0 = p.key0;
            a.key1 = p.key1;
            if (e->axis_z)
                checker_pass_kernel<double, true><<<grid, block, 0, st>>>(a, c, hsel, pass);
            else
                checker_pass_kernel<double, false><<<grid, block, 0, st>>>(a, c, hsel, pass);
        } else {
            PairArgs a = pair_args(e, p, b, hsel);
            a.sw = ctl(pass);
            const bool sw = a.sw.mode != 0;
            if (e->bx == 0) {
                auto fn = e->axis_z ? (sw ? checker_pair_tiled_kernel<true, true> : checker_pair_tiled_kernel<true, false>)
                                    : (sw ? checker_pair_tiled_kernel<false, true> : checker_pair_tiled_kernel<false, false>);
                fn<<<e->tile_grid, 256, e->tile_smem, st>>>(a, e->tile, c, hsel, pass);
            } else {
                const dim3 pgrid(a.nkx * ((a.Ly2 + rby - 1) / rby), e->shape[2], e->n_inst);
                auto fn = pair_kernel_fn(e->axis_z, sw, pair_cell_mode(a));
                if (sw) {
                    // one block per (row block, z, instance) for the leading pass; the
                    // trailing pass, often skipped, on a persistent grid of 8 CTAs a SM
                    const uint64_t nvb = uint64_t(pgrid.x) * pgrid.y * pgrid.z;
                    const uint64_t cap = a.sw.mode == 2 ? uint64_t(e->sm_count > 0 ? e->sm_count : 148) * 8 : nvb;
                    fn<<<static_cast<unsigned>(std::min(nvb, cap)), block, 0, st>>>(a, c, hsel, pass);
                } else {
                    fn<<<pgrid, block, 0, st>>>(a, c, hsel, pass);
                }
            }
        }
        err = cudaGetLastError();
        ++*kernels;
    }
    if (err == cudaSuccess && ev1) err = cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    // the TTM branch joins after the passes' end mark
    if (ttm_beside && err == cudaSuccess) err = cudaStreamWaitEvent(st, e->ev_ttm, 0);
    bool partials = false;
    if (err == cudaSuccess && p.sample_every > 0 && !p.obs_skip) {
        if (e->pair) {
            // observables straight from the pair layout (sampling steps only)
            err = engine_obs_partials(e, p, b, 0, st);
            partials = true;
        } else {
            const int bs = 256;
            const int64_t gs = (e->n_total + bs - 1) / bs;
            to_general_kernel<double><<<gs, bs, 0, st>>>(static_cast<const double4a *>(e->S),
                                                         static_cast<double *>(b.sx), static_cast<double *>(b.sy),
                                                         static_cast<double *>(b.sz), e->n_total, b.step,
                                                         p.sample_every, 1);
            err = cudaGetLastError();
        }
        ++*kernels;
    }
    // (with the TTM beside the passes: only the observables or the bare step increment)
    if (err == cudaSuccess)
        err = step_tail(p, b, tp, ttm_active && !ttm_beside, p.n_instances, e->precision, p.obs_blocks, st, kernels,
                        partials);
    return err;
}

cudaError_t engine_run_steps(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                             bool ttm_active, int64_t nsteps, cudaStream_t st, int *kernels, cudaEvent_t ev0,
                             cudaEvent_t ev1)
{
    *kernels = 0;
    if (e->engine != TTS_ENGINE_RESIDENT) return cudaErrorNotSupported;
    cudaError_t err = cudaSuccess;
    if (ev0) err = cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal);
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
        a.merged = p.merged;
        a.tp = tp;
    };
    // chunks of at most traj_cap steps: the bath trajectory of every instance,
    // then the spin kernel over the chunk, then the step counter
    for (int64_t done = 0; done < nsteps && err == cudaSuccess;) {
        const int chunk = static_cast<int>(std::min<int64_t>(nsteps - done, e->traj_cap));
        const int tb = 128, tg = (e->n_inst + tb - 1) / tb;
        auto chunk_args = [&](auto &a) {
            a.open_state = e->open_state;
            a.first_chunk = done == 0 ? 1 : 0;
            a.last_chunk = done + chunk == nsteps ? 1 : 0;
        };
        if (e->precision == 64) {
            ResArgs<double> a{};
            a.sx = static_cast<double *>(b.sx);
            a.sy = static_cast<double *>(b.sy);
            a.sz = static_cast<double *>(b.sz);
            fill(a);
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spd[t];
            a.traj_sig = static_cast<double *>(e->traj_sig);
            a.traj_T = e->traj_T;
            a.traj_cap = e->traj_cap;
            chunk_args(a);
            resident_traj_kernel<double><<<tg, tb, 0, st>>>(a, chunk);
            if (e->axis_z)
                resident_kernel<double, true><<<e->grid, e->block, e->smem, st>>>(a, chunk);
            else
                resident_kernel<double, false><<<e->grid, e->block, e->smem, st>>>(a, chunk);
        } else {
            ResArgs<float> a{};
            a.sx = static_cast<float *>(b.sx);
            a.sy = static_cast<float *>(b.sy);
            a.sz = static_cast<float *>(b.sz);
            fill(a);
            for (int t = 0; t < TTS_MAX_SPECIES; ++t) a.sp[t] = e->spf[t];
            a.pk = make_pair_consts(e, p, 0);
            a.rk = philox_round_keys(p.key0, p.key1);
            a.traj_sig = static_cast<float *>(e->traj_sig);
            a.traj_T = e->traj_T;
            a.traj_cap = e->traj_cap;
            chunk_args(a);
            resident_traj_kernel<float><<<tg, tb, 0, st>>>(a, chunk);
            if (e->axis_z)
                resident_kernel<float, true><<<e->grid, e->block, e->smem, st>>>(a, chunk);
            else
                resident_kernel<float, false><<<e->grid, e->block, e->smem, st>>>(a, chunk);
        }
        err = cudaGetLastError();
        if (err == cudaSuccess) {
            advance_step_kernel<<<1, 1, 0, st>>>(b.step, chunk, e->queue);
            err = cudaGetLastError();
        }
        *kernels += 3;
        done += chunk;
    }
    if (err == cudaSuccess && ev1) err = cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    return err;
}

int engine_set_cells(EngineState *e, const std::vector<DevInstance> &dinst, const std::vector<int> &cellmap,
                     cudaStream_t)
{
    e->dinst = dinst;
    if (e->engine == TTS_ENGINE_CHECKER) check_cell_formula(e, dinst, cellmap);
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
        launch_pair_to_general(e, b, st, 0, 0);
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
    else {
        const int64_t np = e->n_total / 2;
        pair_from_general_kernel<<<(np + bs - 1) / bs, bs, 0, st>>>(
            static_cast<float4 *>(e->S), static_cast<float4 *>(e->S1), e->cur, static_cast<const float *>(b.sx),
            static_cast<const float *>(b.sy),
            static_cast<const float *>(b.sz), b.species, np, e->shape[0] / 2, e->shape[1] / 2,
            static_cast<uint32_t>(e->n_total / e->n_inst / 4));
    }
    return cudaGetLastError();
}

}  // namespace tts
