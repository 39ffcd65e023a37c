// tts_build.cpp -- host-side construction of one instance: lattice sites,
// random alloy placement (paper Sec. II.D), neighbour lists with J(r)
// (Sec. II.E) and the colour classes that replace the sequential spin sweep.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "tts_internal.h"
#include "tts_philox.cuh"

namespace tts {
namespace {

// Basis vectors in units of a/2 (so all lattice coordinates are integers).
const int kBasisHalf[3][4][3] = {
    {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}},          // sc
    {{0, 0, 0}, {1, 1, 1}, {0, 0, 0}, {0, 0, 0}},          // bcc
    {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}},          // fcc
};
const int kBasisCount[3] = {1, 2, 4};

double exchange_value(const tts_exchange &e, double r)
{
    if (e.kind == TTS_EXCH_NONE || !(r < e.rc)) return 0.0;
    if (e.kind == TTS_EXCH_CONST) return e.J1;
    const double x = (r / e.J3) * (r / e.J3);
    return 4.0 * e.J1 * x * (1.0 - e.J2 * x) * std::exp(-x);
}

double largest_cutoff(const tts_system_desc &d)
{
    double rc = 0.0;
    for (int a = 0; a < d.nspecies; ++a)
        for (int b = 0; b < d.nspecies; ++b)
            if (d.exch[a][b].kind != TTS_EXCH_NONE) rc = std::max(rc, d.exch[a][b].rc);
    return rc;
}

// Exactly round(frac1 * n) sites of species 1, chosen by a partial
// Fisher-Yates shuffle; each swap index is an unbiased bounded integer drawn
// by rejection from Philox words (counter: k, attempt, placement stream, inst).
void place(const tts_system_desc &d, int inst, HostInstance *hi)
{
    const int64_t n = hi->n;
    hi->species.assign(n, 0);
    if (d.nspecies < 2) return;
    const int64_t count = static_cast<int64_t>(std::floor(hi->frac1 * static_cast<double>(n) + 0.5));
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    const uint32_t k0 = static_cast<uint32_t>(d.seed & 0xffffffffu);
    const uint32_t k1 = static_cast<uint32_t>(d.seed >> 32);
    for (int64_t k = 0; k < count; ++k) {
        const uint64_t span = static_cast<uint64_t>(n - k);
        const uint64_t accept_below = (0x100000000ull / span) * span;   // <= 2^32
        uint32_t attempt = 0;
        uint64_t draw;
        do {
            u32x4 c{static_cast<uint32_t>(k), attempt++, kStreamPlacement,
                    static_cast<uint32_t>(d.instance_base + inst)};
            draw = philox4x32_10(c, k0, k1).x;
        } while (draw >= accept_below);
        std::swap(order[k], order[k + static_cast<int64_t>(draw % span)]);
    }
    for (int64_t k = 0; k < count; ++k) hi->species[order[k]] = 1;
}

struct StencilEntry {
    int dcell[3];
    int basis_to;
    double r;
};

void neighbours_lattice(const tts_system_desc &d, HostInstance *hi)
{
    const int lat = d.lattice, nb = kBasisCount[lat];
    const double rc = largest_cutoff(d);
    const int reach = static_cast<int>(std::ceil(rc / d.a)) + 1;
    // per source basis: all lattice offsets closer than the largest cutoff
    std::vector<std::vector<StencilEntry>> stencil(nb);
    for (int b = 0; b < nb; ++b)
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dx = -reach; dx <= reach; ++dx)
                    for (int b2 = 0; b2 < nb; ++b2) {
                        const int hx = 2 * dx + kBasisHalf[lat][b2][0] - kBasisHalf[lat][b][0];
                        const int hy = 2 * dy + kBasisHalf[lat][b2][1] - kBasisHalf[lat][b][1];
                        const int hz = 2 * dz + kBasisHalf[lat][b2][2] - kBasisHalf[lat][b][2];
                        const double r = 0.5 * d.a * std::sqrt(double(hx * hx + hy * hy + hz * hz));
                        if (r > 0.0 && r < rc) stencil[b].push_back({{dx, dy, dz}, b2, r});
                    }
    const int *L = hi->cells;
    hi->nbr_begin.assign(hi->n + 1, 0);
    hi->nbr.clear();
    hi->nbr_J.clear();
    std::vector<std::pair<int64_t, double>> row;
    for (int64_t i = 0; i < hi->n; ++i) {
        const int b = static_cast<int>(i % nb);
        const int64_t cell = i / nb;
        const int ix = static_cast<int>(cell % L[0]);
        const int iy = static_cast<int>((cell / L[0]) % L[1]);
        const int iz = static_cast<int>(cell / (int64_t(L[0]) * L[1]));
        row.clear();
        for (const StencilEntry &e : stencil[b]) {
            const int jx = ((ix + e.dcell[0]) % L[0] + L[0]) % L[0];
            const int jy = ((iy + e.dcell[1]) % L[1] + L[1]) % L[1];
            const int jz = ((iz + e.dcell[2]) % L[2] + L[2]) % L[2];
            const int64_t j = ((int64_t(jz) * L[1] + jy) * L[0] + jx) * nb + e.basis_to;
            const double J = exchange_value(d.exch[hi->species[i]][hi->species[j]], e.r);
            if (J != 0.0) row.emplace_back(j, J);
        }
        std::sort(row.begin(), row.end());
        for (auto &p : row) {
            hi->nbr.push_back(static_cast<int>(p.first));
            hi->nbr_J.push_back(p.second);
        }
        hi->nbr_begin[i + 1] = static_cast<int64_t>(hi->nbr.size());
    }
}

void neighbours_cluster(const tts_system_desc &d, HostInstance *hi)
{
    const double rc = largest_cutoff(d);
    hi->nbr_begin.assign(hi->n + 1, 0);
    hi->nbr.clear();
    hi->nbr_J.clear();
    for (int64_t i = 0; i < hi->n; ++i) {
        for (int64_t j = 0; j < hi->n; ++j) {
            if (j == i) continue;
            double r2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double v = hi->pos[3 * j + k] - hi->pos[3 * i + k];
                r2 += v * v;
            }
            const double r = std::sqrt(r2);
            if (!(r < rc)) continue;
            const double J = exchange_value(d.exch[hi->species[i]][hi->species[j]], r);
            if (J == 0.0) continue;
            hi->nbr.push_back(static_cast<int>(j));
            hi->nbr_J.push_back(J);
        }
        hi->nbr_begin[i + 1] = static_cast<int64_t>(hi->nbr.size());
    }
}

// Graph of the colouring: CSR adjacency, ascending neighbour ids.
struct ColourGraph {
    std::vector<int64_t> begin;
    std::vector<int> adj;
};

// Every pair closer than rc (geometric, periodic lattice or open cluster).
ColourGraph pairs_within(const tts_system_desc &d, const HostInstance &hi, double rc)
{
    ColourGraph g;
    g.begin.assign(hi.n + 1, 0);
    std::vector<int64_t> row;
    if (d.lattice == TTS_LATTICE_CLUSTER) {
        for (int64_t i = 0; i < hi.n; ++i) {
            for (int64_t j = 0; j < hi.n; ++j) {
                if (j == i) continue;
                double r2 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double v = hi.pos[3 * j + k] - hi.pos[3 * i + k];
                    r2 += v * v;
                }
                if (std::sqrt(r2) < rc) g.adj.push_back(static_cast<int>(j));
            }
            g.begin[i + 1] = static_cast<int64_t>(g.adj.size());
        }
        return g;
    }
    const int lat = d.lattice, nb = kBasisCount[lat];
    const int reach = static_cast<int>(std::ceil(rc / d.a)) + 1;
    std::vector<std::vector<StencilEntry>> stencil(nb);
    for (int b = 0; b < nb; ++b)
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dx = -reach; dx <= reach; ++dx)
                    for (int b2 = 0; b2 < nb; ++b2) {
                        const int hx = 2 * dx + kBasisHalf[lat][b2][0] - kBasisHalf[lat][b][0];
                        const int hy = 2 * dy + kBasisHalf[lat][b2][1] - kBasisHalf[lat][b][1];
                        const int hz = 2 * dz + kBasisHalf[lat][b2][2] - kBasisHalf[lat][b][2];
                        const double r = 0.5 * d.a * std::sqrt(double(hx * hx + hy * hy + hz * hz));
                        if (r > 0.0 && r < rc) stencil[b].push_back({{dx, dy, dz}, b2, r});
                    }
    const int *L = hi.cells;
    for (int64_t i = 0; i < hi.n; ++i) {
        const int b = static_cast<int>(i % nb);
        const int64_t cell = i / nb;
        const int ix = static_cast<int>(cell % L[0]);
        const int iy = static_cast<int>((cell / L[0]) % L[1]);
        const int iz = static_cast<int>(cell / (int64_t(L[0]) * L[1]));
        row.clear();
        for (const StencilEntry &e : stencil[b]) {
            const int jx = ((ix + e.dcell[0]) % L[0] + L[0]) % L[0];
            const int jy = ((iy + e.dcell[1]) % L[1] + L[1]) % L[1];
            const int jz = ((iz + e.dcell[2]) % L[2] + L[2]) % L[2];
            const int64_t j = ((int64_t(jz) * L[1] + jy) * L[0] + jx) * nb + e.basis_to;
            if (j != i) row.push_back(j);
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        for (int64_t j : row) g.adj.push_back(static_cast<int>(j));
        g.begin[i + 1] = static_cast<int64_t>(g.adj.size());
    }
    return g;
}

bool proper(const ColourGraph &g, int64_t n, const std::vector<int> &col)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = g.begin[i]; k < g.begin[i + 1]; ++k)
            if (col[g.adj[k]] == col[i]) return false;
    return true;
}

// position on a cycle of length L mapped to Z_3 so that neighbours differ by
// +-1 (mod 3), wrap included: x mod 3, except the last site when L = 1 mod 3
int ring3(int x, int L) { return (L % 3 == 1 && x == L - 1) ? 1 : x % 3; }

}  // namespace

void colour_instance(const tts_system_desc &d, HostInstance *hi)
{
    const int64_t n = hi->n;
    hi->colour.assign(n, 0);
    if (hi->nbr.empty()) {
        hi->ncolours = 1;
        return;
    }
    // the graph to colour: exchange neighbours, or every pair within colour_rc
    ColourGraph g;
    if (d.colour_rc > largest_cutoff(d)) {
        g = pairs_within(d, *hi, d.colour_rc);
    } else {
        g.begin = hi->nbr_begin;
        g.adj = hi->nbr;
    }
    if (d.lattice != TTS_LATTICE_CLUSTER) {
        const int nb = kBasisCount[d.lattice];
        const int *L = hi->cells;
        const bool all_even = (L[0] % 2 == 0) && (L[1] % 2 == 0) && (L[2] % 2 == 0);
        std::vector<int> rule(n);
        for (int64_t i = 0; i < n; ++i) {
            const int b = static_cast<int>(i % nb);
            const int64_t cell = i / nb;
            const int ix = static_cast<int>(cell % L[0]);
            const int iy = static_cast<int>((cell / L[0]) % L[1]);
            const int iz = static_cast<int>(cell / (int64_t(L[0]) * L[1]));
            const int parity = (ix + iy + iz) & 1;
            if (d.lattice == TTS_LATTICE_SC)
                rule[i] = all_even ? parity : (ring3(ix, L[0]) + ring3(iy, L[1]) + ring3(iz, L[2])) % 3;
            else if (d.lattice == TTS_LATTICE_BCC)
                rule[i] = 2 * b + parity;
            else
                rule[i] = b;
        }
        if (proper(g, n, rule)) {
            hi->colour = rule;
            hi->ncolours = d.lattice == TTS_LATTICE_SC ? (all_even ? 2 : 3) : 4;
            return;
        }
    }
    // greedy, ascending atom id
    std::vector<int64_t> seen(n + 1, -1);
    int used = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = g.begin[i]; k < g.begin[i + 1]; ++k)
            if (g.adj[k] < i) seen[hi->colour[g.adj[k]]] = i;
        int c = 0;
        while (seen[c] == i) ++c;
        hi->colour[i] = c;
        used = std::max(used, c + 1);
    }
    hi->ncolours = used;
}

int build_instance(const tts_system_desc &d, int inst, HostInstance *hi, std::string *err)
{
    char msg[256];
    if (d.lattice == TTS_LATTICE_CLUSTER) {
        if (d.n_explicit < 1 || !d.pos_explicit) {
            *err = "cluster needs n_explicit >= 1 and positions";
            return TTS_ERR_ARG;
        }
        hi->n = d.n_explicit;
        hi->nbasis = 1;
        hi->pos.assign(d.pos_explicit, d.pos_explicit + 3 * hi->n);
        hi->species.assign(hi->n, 0);
        for (int64_t i = 0; i < hi->n; ++i) {
            const int t = d.species_explicit ? d.species_explicit[i] : 0;
            if (t < 0 || t >= d.nspecies) {
                *err = "cluster species out of range";
                return TTS_ERR_ARG;
            }
            hi->species[i] = static_cast<uint8_t>(t);
        }
        neighbours_cluster(d, hi);
        colour_instance(d, hi);
        return TTS_OK;
    }
    if (d.lattice < 0 || d.lattice > 2) {
        *err = "unknown lattice";
        return TTS_ERR_ARG;
    }
    for (int k = 0; k < 3; ++k) {
        hi->cells[k] = d.inst_cells ? d.inst_cells[3 * inst + k] : (&d.nx)[k];
        if (hi->cells[k] < 1) {
            *err = "cell counts must be >= 1";
            return TTS_ERR_ARG;
        }
    }
    hi->frac1 = d.inst_frac1 ? d.inst_frac1[inst] : d.frac1;
    if (!(hi->frac1 >= 0.0 && hi->frac1 <= 1.0)) {
        *err = "species-1 fraction outside [0, 1]";
        return TTS_ERR_ARG;
    }
    const int nb = kBasisCount[d.lattice];
    hi->nbasis = nb;
    hi->n = int64_t(hi->cells[0]) * hi->cells[1] * hi->cells[2] * nb;
    if (hi->n > 0x7fffffffLL) {
        *err = "instance too large for 32-bit atom ids";
        return TTS_ERR_ARG;
    }
    const double rc = largest_cutoff(d);
    for (int k = 0; k < 3; ++k) {
        hi->box[k] = hi->cells[k] * d.a;
        if (!(hi->box[k] > 2.0 * rc)) {
            std::snprintf(msg, sizeof msg, "instance %d: box edge %d (%.4f A) must exceed twice the cutoff (%.4f A)",
                          inst, k, hi->box[k], rc);
            *err = msg;
            return TTS_ERR_ARG;
        }
    }
    hi->half.resize(3 * hi->n);
    hi->pos.resize(3 * hi->n);
    for (int64_t i = 0; i < hi->n; ++i) {
        const int b = static_cast<int>(i % nb);
        const int64_t cell = i / nb;
        const int c[3] = {static_cast<int>(cell % hi->cells[0]),
                          static_cast<int>((cell / hi->cells[0]) % hi->cells[1]),
                          static_cast<int>(cell / (int64_t(hi->cells[0]) * hi->cells[1]))};
        for (int k = 0; k < 3; ++k) {
            hi->half[3 * i + k] = 2 * c[k] + kBasisHalf[d.lattice][b][k];
            hi->pos[3 * i + k] = 0.5 * d.a * hi->half[3 * i + k];
        }
    }
    place(d, inst, hi);
    neighbours_lattice(d, hi);
    colour_instance(d, hi);
    return TTS_OK;
}

}  // namespace tts
