/*
 * tts_oracle.c -- plain FP64 CPU oracle of the stochastic spin advance.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke entry
 * and the benchmark's CPU-baseline leg may load, call or run this file.  It
 * shares no code, header, table or constant with the CUDA library, and it is
 * written for a reader checking it against the paper by eye: one atom at a
 * time, in canonical atom order, in double precision, with no blocking,
 * fusion or reordering beyond what the method states.
 *
 * What it computes (paper sections / equations):
 *  - Eq. 1: the LLG equation ds/dt = -(1/(1+a^2)) [s x w + a s x (s x w)],
 *    written in SI as w = gamma B with B the effective field in tesla.
 *  - Sec. II.C: deterministic field B_i = -(1/mu_i) dH/ds_i (the 1/mu_i
 *    prefactor of fix moment/scale/spin) and a noise field whose amplitude
 *    scales as 1/sqrt(mu_i) (the mu_fdt option), i.e. the FDT variance
 *    2 alpha k_B T / (gamma mu_i h) for a sub-step of length h.
 *  - Eq. 2 / Sec. II.B: the bath temperature of atom i is the electron
 *    temperature of the TTM grid cell that holds atom i.
 *  - Sec. II.E: the Bethe-Slater radial exchange J(r) = 4 J1 x (1 - J2 x) e^-x,
 *    x = (r/J3)^2, and the re-derivation of (J2, J3) for a new lattice.
 *  - Sec. II.A: the symplectic Suzuki-Trotter splitting, taken as a symmetric
 *    sweep over colour classes (colours ascending at h = dt/2, the last colour
 *    at h = dt, colours descending at h = dt/2).
 *  - Sec. II.D: random alloy placement by sampling sites without replacement.
 *  - Sec. II.B (fix ttm): the two-temperature model grid with a laser source.
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes): the per-spin sub-step is the exact LLG flow under the field frozen at
 * the start of the sub-step, with its on-site anisotropy part taken at the
 * predicted midpoint (substep_field); noise is Philox4x32-10 + Box-Muller keyed by
 * (atom, step, pass, instance); the spin bath reads T_e(t_n) for the whole
 * step; the coupling from spins back to T_e is absent (one-way).
 */
#include "tts_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 values, SI */
static const double KB = 1.380649e-23;       /* J/K */
static const double MUB = 9.2740100783e-24;  /* J/T */
static const double GAMMA = 1.76085963023e11;/* rad s^-1 T^-1 */
static const double ANG = 1e-10;             /* m */
static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the description in Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11: ten rounds of two   */
/* 32x32->64 multiplies with the counter words permuted and xored with the   */
/* key, the key advanced by the Weyl constants between rounds.               */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23 random bits plus one half-bit: (2k+1) * 2^-24 with k < 2^23 has at most
 * 24 significant bits, so the value is exact in float32 as well as float64. */
double orc_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Box-Muller: g1, g2 from (u0, u1); g3 from (u2, u3). */
void orc_gauss3(const uint32_t w[4], double g[3])
{
    double u0 = orc_uniform(w[0]), u1 = orc_uniform(w[1]);
    double u2 = orc_uniform(w[2]), u3 = orc_uniform(w[3]);
    double r01 = sqrt(-2.0 * log(u0));
    double r23 = sqrt(-2.0 * log(u2));
    g[0] = r01 * cos(2.0 * PI * u1);
    g[1] = r01 * sin(2.0 * PI * u1);
    g[2] = r23 * cos(2.0 * PI * u3);
}

/* ------------------------------------------------------------------------- */
/* Exchange function, Sec. II.E                                              */
/* ------------------------------------------------------------------------- */
double orc_bethe_slater(double r, double J1, double J2, double J3)
{
    double x = (r / J3) * (r / J3);
    return 4.0 * J1 * x * (1.0 - J2 * x) * exp(-x);
}

/* dJ/dr = dJ/dx * dx/dr with dJ/dx = 4 J1 e^-x (1 - 2 J2 x - x + J2 x^2)
 * and dx/dr = 2 r / J3^2. */
double orc_bethe_slater_deriv(double r, double J1, double J2, double J3)
{
    double x = (r / J3) * (r / J3);
    double dJdx = 4.0 * J1 * exp(-x) * (1.0 - 2.0 * J2 * x - x + J2 * x * x);
    return dJdx * 2.0 * r / (J3 * J3);
}

/* Sec. II.E: (1) dJ/dx = 0 at x1 gives J2 = (x1 - 1) / (x1 (x1 - 2));
 * (2) J(x1) = J1 gives 4 x1 (1 - J2 x1) e^-x1 = 1.  Substituting (1) into (2)
 * leaves one equation in x1, solved here by bisection on (0, 1) where the
 * extremum is a maximum of a ferromagnetic J; then J3 = r1 / sqrt(x1). */
static double rederive_residual(double x)
{
    double J2 = (x - 1.0) / (x * (x - 2.0));
    return 4.0 * x * (1.0 - J2 * x) * exp(-x) - 1.0;
}

int orc_rederive_exchange(double r1, double *x1, double *J2, double *J3)
{
    double lo = 1e-6, hi = 1.0 - 1e-12;
    double flo = rederive_residual(lo), fhi = rederive_residual(hi);
    if (flo * fhi > 0.0) return -1;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = rederive_residual(mid);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    double x = 0.5 * (lo + hi);
    *x1 = x;
    *J2 = (x - 1.0) / (x * (x - 2.0));
    *J3 = r1 / sqrt(x);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact single-spin flow of Eq. 1 under a field held fixed for time h.      */
/* With w = gamma |B| / (1 + alpha^2) and polar angle theta measured from    */
/* the field direction, Eq. 1 gives d(phi)/dt = w (counter-clockwise about   */
/* +B) and d(theta)/dt = -alpha w sin(theta), whose solution is              */
/* tan(theta/2) = tan(theta0/2) exp(-alpha w t).                             */
/* ------------------------------------------------------------------------- */
void orc_flow(double s[3], const double Bf[3], double alpha, double h)
{
    double Bm = sqrt(Bf[0] * Bf[0] + Bf[1] * Bf[1] + Bf[2] * Bf[2]);
    if (!(Bm > 0.0)) return;
    double b[3] = {Bf[0] / Bm, Bf[1] / Bm, Bf[2] / Bm};
    double c = s[0] * b[0] + s[1] * b[1] + s[2] * b[2];
    double p[3] = {s[0] - c * b[0], s[1] - c * b[1], s[2] - c * b[2]};
    double pm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (pm <= 1e-300) return;  /* spin along the field: a fixed point */
    double e1[3] = {p[0] / pm, p[1] / pm, p[2] / pm};
    double e2[3] = {b[1] * e1[2] - b[2] * e1[1],
                    b[2] * e1[0] - b[0] * e1[2],
                    b[0] * e1[1] - b[1] * e1[0]};
    /* tan(theta0/2) from (c, pm) without cancellation */
    double u0 = (c >= 0.0) ? pm / (1.0 + c) : (1.0 - c) / pm;
    double w = GAMMA * Bm / (1.0 + alpha * alpha);
    double u = u0 * exp(-alpha * w * h);
    double cn = (1.0 - u * u) / (1.0 + u * u);
    double sn = 2.0 * u / (1.0 + u * u);
    double phi = w * h;
    double cp = cos(phi), sp = sin(phi);
    double out[3];
    for (int k = 0; k < 3; ++k)
        out[k] = cn * b[k] + sn * (cp * e1[k] + sp * e2[k]);
    double nrm = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    for (int k = 0; k < 3; ++k) s[k] = out[k] / nrm;
}

/* ------------------------------------------------------------------------- */
/* System                                                                    */
/* ------------------------------------------------------------------------- */
struct orc_sys {
    orc_params p;
    int n;                 /* atoms */
    int periodic;          /* 1 for lattices 0..2 */
    double box[3];         /* angstrom */
    double *pos;           /* 3n, angstrom */
    int *ipos2;            /* 3n, position in units of a/2 (lattices 0..2) */
    int *species;          /* n */
    int *colour;           /* n */
    int ncolours;
    int *nbr_start;        /* n+1 */
    int *nbr_j;            /* neighbour ids, ascending per atom */
    double *nbr_J;         /* J_ij, J */
    double *s;             /* 3n unit spins */
    int64_t step;
    /* TTM */
    int has_ttm;
    orc_ttm t;
    int nc;                /* cells */
    double *Te, *Tl;
    double *scratch;       /* 2 nc: per-sub-step increments */
    int *cell_of;          /* n */
    double cellvol;        /* m^3 */
    double dxc[3];         /* m */
    double *src_shape;     /* nc */
    int substeps;
    double P0;
    double src_energy;     /* J deposited so far (integral of S dV dt) */
    /* samples */
    double *samples;
    int64_t nsamp, capsamp;
    /* moving lattice */
    int lattice_on;
    orc_lattice L;
    double mass;           /* kg */
    double *vel;           /* 3n, m/s */
    double *force;         /* 3n, N (Morse + magnetic) */
    int *mor_start, *mor_j;/* Morse pair list, ascending j */
    int64_t lstep;
    int colour_violations;
    double ion_to_e;       /* energy handed from ions to electrons, J */
};

static double sq(double x) { return x * x; }
static void rebuild_lists(orc_sys *S);

static const double BASIS_SC[1][3] = {{0, 0, 0}};
static const double BASIS_BCC[2][3] = {{0, 0, 0}, {0.5, 0.5, 0.5}};
static const double BASIS_FCC[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};

static int basis_count(int lattice)
{
    return lattice == 0 ? 1 : lattice == 1 ? 2 : 4;
}

static const double *basis_vec(int lattice, int b)
{
    return lattice == 0 ? BASIS_SC[b] : lattice == 1 ? BASIS_BCC[b] : BASIS_FCC[b];
}

/* minimum-image distance vector j - i (angstrom) */
static void min_image(const orc_sys *S, int i, int j, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        double v = S->pos[3 * j + k] - S->pos[3 * i + k];
        if (S->periodic) {
            double L = S->box[k];
            v -= L * floor(v / L + 0.5);
        }
        d[k] = v;
    }
}

static double pair_J(const orc_params *p, int ti, int tj, double r)
{
    const orc_exch *e = &p->exch[ti][tj];
    if (e->kind == 0 || r >= e->rc) return 0.0;
    if (e->kind == 1) return e->J1;
    return orc_bethe_slater(r, e->J1, e->J2, e->J3);
}

static double max_rc(const orc_params *p)
{
    double rc = 0.0;
    for (int a = 0; a < p->nspecies; ++a)
        for (int b = 0; b < p->nspecies; ++b)
            if (p->exch[a][b].kind != 0 && p->exch[a][b].rc > rc) rc = p->exch[a][b].rc;
    return rc;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Neighbour list: every j != i within the largest cutoff, by minimum image,
 * ascending j.  Lattices: candidates from the cells within ceil(rc/a) of the
 * atom's cell (a site in cell c + d is at least (|d_k| - 1) a away along axis
 * k, so nothing closer than rc lies further out); clusters: all pairs.
 * Pairs whose J is zero for their species are kept out. */
static int build_neighbours(orc_sys *S, char *err, int errlen)
{
    double rc = max_rc(&S->p);
    int n = S->n;
    int cap = 16, *tmp = malloc(sizeof(int) * cap);
    S->nbr_start = malloc(sizeof(int) * (n + 1));
    int total = 0, totcap = n * 8 + 16;
    S->nbr_j = malloc(sizeof(int) * totcap);
    S->nbr_J = malloc(sizeof(double) * totcap);
    int nb = S->p.lattice <= 2 ? basis_count(S->p.lattice) : 1;
    int R = S->p.lattice <= 2 ? (int)ceil(rc / S->p.a) : 0;
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        if (S->p.lattice <= 2) {
            int cell = i / nb;
            int ix = cell % S->p.nx, iy = (cell / S->p.nx) % S->p.ny, iz = cell / (S->p.nx * S->p.ny);
            for (int dz = -R; dz <= R; ++dz)
                for (int dy = -R; dy <= R; ++dy)
                    for (int dx = -R; dx <= R; ++dx)
                        for (int b2 = 0; b2 < nb; ++b2) {
                            int jx = ((ix + dx) % S->p.nx + S->p.nx) % S->p.nx;
                            int jy = ((iy + dy) % S->p.ny + S->p.ny) % S->p.ny;
                            int jz = ((iz + dz) % S->p.nz + S->p.nz) % S->p.nz;
                            int j = ((jz * S->p.ny + jy) * S->p.nx + jx) * nb + b2;
                            if (j == i) continue;
                            double d[3];
                            min_image(S, i, j, d);
                            if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) >= rc) continue;
                            if (cnt == cap) { cap *= 2; tmp = realloc(tmp, sizeof(int) * cap); }
                            tmp[cnt++] = j;
                        }
        } else {
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (cnt == cap) { cap *= 2; tmp = realloc(tmp, sizeof(int) * cap); }
                tmp[cnt++] = j;
            }
        }
        qsort(tmp, cnt, sizeof(int), cmp_int);
        S->nbr_start[i] = total;
        int last = -1;
        for (int k = 0; k < cnt; ++k) {
            int j = tmp[k];
            if (j == last) continue;
            last = j;
            double d[3];
            min_image(S, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r >= rc) continue;
            double J = pair_J(&S->p, S->species[i], S->species[j], r);
            if (J == 0.0) continue;
            if (total == totcap) {
                totcap *= 2;
                S->nbr_j = realloc(S->nbr_j, sizeof(int) * totcap);
                S->nbr_J = realloc(S->nbr_J, sizeof(double) * totcap);
            }
            S->nbr_j[total] = j;
            S->nbr_J[total] = J;
            ++total;
        }
    }
    S->nbr_start[n] = total;
    free(tmp);
    (void)err; (void)errlen;
    return 0;
}

/* Colouring (replaces the sequential sector sweep).  Lattice rules, each used
 * only when it is a proper colouring of the neighbour graph:
 *   sc, all edges even: parity (ix+iy+iz) mod 2                  (2 colours)
 *   sc, otherwise:      (f(ix)+f(iy)+f(iz)) mod 3                (3 colours)
 *                       with f(x) = x mod 3 on a cycle of length L, except
 *                       f(L-1) = 1 when L mod 3 == 1, so that f changes by +-1
 *                       (mod 3) across every edge including the wrap
 *   bcc:                2 * basis + parity                      (4 colours)
 *   fcc:                basis index                             (4 colours)
 * otherwise greedy colouring in ascending atom id (each atom takes the smallest
 * colour unused by its already-coloured neighbours).  No neighbours at all:
 * a single colour. */
static int colouring_valid(int n, const int *start, const int *adj, const int *col)
{
    for (int i = 0; i < n; ++i)
        for (int k = start[i]; k < start[i + 1]; ++k)
            if (col[adj[k]] == col[i]) return 0;
    return 1;
}

static int cycle3(int x, int L)
{
    if (L % 3 == 1 && x == L - 1) return 1;
    return x % 3;
}

/* The graph to colour: the exchange neighbours, or, with colour_rc above the
 * exchange cutoff, every pair closer than colour_rc (minimum image; all pairs
 * checked). */
static void colour_graph(const orc_sys *S, int **start_out, int **adj_out)
{
    int n = S->n;
    if (!(S->p.colour_rc > max_rc(&S->p))) {
        *start_out = NULL;
        *adj_out = NULL;
        return;
    }
    int *start = malloc(sizeof(int) * (n + 1)), cap = 16 * n + 16, tot = 0;
    int *adj = malloc(sizeof(int) * cap);
    for (int i = 0; i < n; ++i) {
        start[i] = tot;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(S, i, j, d);
            if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < S->p.colour_rc) {
                if (tot == cap) { cap *= 2; adj = realloc(adj, sizeof(int) * cap); }
                adj[tot++] = j;
            }
        }
    }
    start[n] = tot;
    *start_out = start;
    *adj_out = adj;
}

static void build_colours(orc_sys *S)
{
    int n = S->n;
    S->colour = calloc(n, sizeof(int));
    if (S->nbr_start[n] == 0) { S->ncolours = 1; return; }
    int *gs, *ga;
    colour_graph(S, &gs, &ga);
    const int *start = gs ? gs : S->nbr_start, *adj = gs ? ga : S->nbr_j;
    int rule = 0, K = 0;
    if (S->p.lattice <= 2) {
        int nb = basis_count(S->p.lattice);
        int even = (S->p.nx % 2 == 0) && (S->p.ny % 2 == 0) && (S->p.nz % 2 == 0);
        for (int i = 0; i < n; ++i) {
            int b = i % nb, cell = i / nb;
            int ix = cell % S->p.nx, iy = (cell / S->p.nx) % S->p.ny, iz = cell / (S->p.nx * S->p.ny);
            int par = (ix + iy + iz) & 1;
            if (S->p.lattice == 0)
                S->colour[i] = even ? par
                                    : (cycle3(ix, S->p.nx) + cycle3(iy, S->p.ny) + cycle3(iz, S->p.nz)) % 3;
            else if (S->p.lattice == 1) S->colour[i] = 2 * b + par;
            else S->colour[i] = b;
        }
        K = S->p.lattice == 0 ? (even ? 2 : 3) : 4;
        rule = colouring_valid(n, start, adj, S->colour);
    }
    if (rule) {
        S->ncolours = K;
    } else {
        int maxc = 0;
        int *used = calloc(n + 1, sizeof(int));
        for (int i = 0; i < n; ++i) S->colour[i] = -1;
        for (int i = 0; i < n; ++i) {
            for (int k = start[i]; k < start[i + 1]; ++k) {
                int c = S->colour[adj[k]];
                if (c >= 0) used[c] = i + 1;
            }
            int c = 0;
            while (used[c] == i + 1) ++c;
            S->colour[i] = c;
            if (c + 1 > maxc) maxc = c + 1;
        }
        free(used);
        S->ncolours = maxc;
    }
    free(gs);
    free(ga);
}

/* Random alloy, Sec. II.D: exactly round(frac1 * N) sites take species 1,
 * chosen by a partial Fisher-Yates shuffle (sampling without replacement).
 * Bounded integers by rejection from Philox words (no modulo bias).
 * Philox counter: (position k, attempt, 0xFFFF0000, instance). */
static void place_species(orc_sys *S)
{
    int n = S->n;
    for (int i = 0; i < n; ++i) S->species[i] = 0;
    if (S->p.nspecies < 2) return;
    long n1 = (long)floor(S->p.frac1 * (double)n + 0.5);
    int *perm = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    uint32_t key[2] = {(uint32_t)(S->p.seed & 0xffffffffu), (uint32_t)(S->p.seed >> 32)};
    for (long k = 0; k < n1; ++k) {
        uint32_t range = (uint32_t)(n - k);
        uint32_t limit = (uint32_t)((4294967296ull / range) * range);
        uint32_t attempt = 0, x;
        for (;;) {
            uint32_t ctr[4] = {(uint32_t)k, attempt, 0xFFFF0000u, S->p.instance}, out[4];
            orc_philox4x32_10(ctr, key, out);
            x = out[0];
            ++attempt;
            if (limit == 0 || x < limit) break;   /* limit == 0 only if range divides 2^32 */
        }
        long j = k + (long)(x % range);
        int t = perm[k]; perm[k] = perm[j]; perm[j] = t;
    }
    for (long k = 0; k < n1; ++k) S->species[perm[k]] = 1;
    free(perm);
}

orc_sys *orc_create(const orc_params *p, char *err, int errlen)
{
    orc_sys *S = calloc(1, sizeof(orc_sys));
    S->p = *p;
    if (p->nspecies < 1 || p->nspecies > 2) {
        snprintf(err, errlen, "nspecies must be 1 or 2");
        free(S);
        return NULL;
    }
    if (p->lattice <= 2) {
        int nb = basis_count(p->lattice);
        S->periodic = 1;
        S->n = p->nx * p->ny * p->nz * nb;
        S->box[0] = p->nx * p->a; S->box[1] = p->ny * p->a; S->box[2] = p->nz * p->a;
        double rc = max_rc(p);
        for (int k = 0; k < 3; ++k)
            if (S->box[k] <= 2.0 * rc) {
                snprintf(err, errlen, "box edge %d (%.3f A) must exceed twice the cutoff", k, S->box[k]);
                free(S);
                return NULL;
            }
        S->pos = malloc(sizeof(double) * 3 * S->n);
        S->ipos2 = malloc(sizeof(int) * 3 * S->n);
        for (int iz = 0; iz < p->nz; ++iz)
            for (int iy = 0; iy < p->ny; ++iy)
                for (int ix = 0; ix < p->nx; ++ix)
                    for (int b = 0; b < nb; ++b) {
                        int i = ((iz * p->ny + iy) * p->nx + ix) * nb + b;
                        const double *bv = basis_vec(p->lattice, b);
                        int c3[3] = {ix, iy, iz};
                        for (int k = 0; k < 3; ++k) {
                            S->ipos2[3 * i + k] = 2 * c3[k] + (int)(2.0 * bv[k]);
                            S->pos[3 * i + k] = (c3[k] + bv[k]) * p->a;
                        }
                    }
        S->species = malloc(sizeof(int) * S->n);
        place_species(S);
    } else {
        S->periodic = 0;
        S->n = p->n_explicit;
        S->pos = malloc(sizeof(double) * 3 * S->n);
        S->species = malloc(sizeof(int) * S->n);
        for (int i = 0; i < S->n; ++i) {
            for (int k = 0; k < 3; ++k) S->pos[3 * i + k] = p->pos_explicit[3 * i + k];
            S->species[i] = p->species_explicit ? p->species_explicit[i] : 0;
        }
    }
    S->p.pos_explicit = NULL;
    S->p.species_explicit = NULL;
    build_neighbours(S, err, errlen);
    build_colours(S);
    S->s = malloc(sizeof(double) * 3 * S->n);
    for (int i = 0; i < S->n; ++i) {
        const double *d = p->init_dir[S->species[i]];
        double m = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) S->s[3 * i + k] = d[k] / m;
    }
    S->step = 0;
    return S;
}

void orc_free(orc_sys *S)
{
    if (!S) return;
    free(S->pos); free(S->ipos2); free(S->species); free(S->colour);
    free(S->nbr_start); free(S->nbr_j); free(S->nbr_J); free(S->s);
    free(S->Te); free(S->Tl); free(S->cell_of); free(S->src_shape); free(S->scratch);
    free(S->samples);
    free(S->vel); free(S->force); free(S->mor_start); free(S->mor_j);
    free(S);
}

/* ------------------------------------------------------------------------- */
/* Two-temperature model grid (fix ttm of Sec. II.B): explicit FTCS update   */
/* of the electron energy density E_e = gamma_e T_e^2 / 2 with a periodic    */
/* 7-point Laplacian, e-ph exchange G (T_e - T_l) and a Gaussian laser       */
/* source S(r, t) = P0 exp(-(t - t0)^2 / (2 sigma_t^2)) f(r).                */
/* ------------------------------------------------------------------------- */
static double pulse_sigma(const orc_ttm *t) { return t->fwhm / (2.0 * sqrt(2.0 * log(2.0))); }
static double pulse_t0(const orc_ttm *t) { return t->t0 >= 0.0 ? t->t0 : 3.0 * pulse_sigma(t); }

static int cidx(const orc_sys *S, int cx, int cy, int cz)
{
    int nx = S->t.ncx, ny = S->t.ncy, nz = S->t.ncz;
    cx = (cx % nx + nx) % nx; cy = (cy % ny + ny) % ny; cz = (cz % nz + nz) % nz;
    return (cz * ny + cy) * nx + cx;
}

/* One TTM advance over Dt from time t_start, in S->substeps equal sub-steps,
 * on the given grids; returns the source energy deposited (J). */
/* use_G = 0 drops the G (T_e - T_l) exchange: with a moving lattice the ions
 * exchange energy with the electrons through their own friction and noise. */
/* The three-stage electron-temperature profile of the paper's GdFeCo runs
 * (Sec. II.D): peak, half the peak, then the base temperature. */
static double profile_Te(const orc_ttm *t, double tt)
{
    if (tt < t->t0) return t->peak_Te;
    if (tt < t->t0 + t->fwhm) return 0.5 * t->peak_Te;
    return t->T0;
}

static double ttm_advance(const orc_sys *S, double *Te, double *Tl, double t_start, double Dt, double P0, int use_G)
{
    const orc_ttm *t = &S->t;
    if (t->source == 3) {
        for (int c = 0; c < S->nc; ++c) { Te[c] = profile_Te(t, t_start + Dt); Tl[c] = t->T0; }
        return 0.0;
    }
    int m = S->substeps;
    double dl = Dt / m;
    double sig = pulse_sigma(t), t0 = pulse_t0(t);
    double *dE = S->scratch, *dT = S->scratch + S->nc;
    double dep = 0.0;
    int nd[3] = {t->ncx, t->ncy, t->ncz};
    for (int k = 0; k < m; ++k) {
        double tt = t_start + k * dl;
        double pulse = (t->source != 0) ? P0 * exp(-sq(tt - t0) / (2.0 * sig * sig)) : 0.0;
        for (int cz = 0; cz < t->ncz; ++cz)
            for (int cy = 0; cy < t->ncy; ++cy)
                for (int cx = 0; cx < t->ncx; ++cx) {
                    int c = cidx(S, cx, cy, cz);
                    double lap = 0.0;
                    int cc[3] = {cx, cy, cz};
                    for (int d = 0; d < 3; ++d) {
                        if (nd[d] < 2) continue;
                        int cp[3] = {cc[0], cc[1], cc[2]}, cm[3] = {cc[0], cc[1], cc[2]};
                        cp[d] += 1; cm[d] -= 1;
                        double Tp = Te[cidx(S, cp[0], cp[1], cp[2])];
                        double Tm = Te[cidx(S, cm[0], cm[1], cm[2])];
                        lap += (Tp - 2.0 * Te[c] + Tm) / (S->dxc[d] * S->dxc[d]);
                    }
                    double src = pulse * S->src_shape[c];
                    double G = use_G ? t->G : 0.0;
                    dE[c] = dl * (t->kappa_e * lap - G * (Te[c] - Tl[c]) + src);
                    dT[c] = dl * G * (Te[c] - Tl[c]) / t->C_l;
                    dep += dl * src * S->cellvol;
                }
        for (int c = 0; c < S->nc; ++c) {
            double Ee = 0.5 * t->gamma_e * Te[c] * Te[c] + dE[c];
            Te[c] = sqrt(2.0 * Ee / t->gamma_e);
            Tl[c] += dT[c];
        }
    }
    return dep;
}

/* Time step of the TTM grid: the spin step, or the lattice step when the
 * lattice moves (the grid then advances once per lattice step). */
static double ttm_dt(const orc_sys *S)
{
    return S->lattice_on ? S->L.spin_substeps * S->p.dt : S->p.dt;
}

/* Peak electron temperature over the step grid t_n of a TTM-only run. */
static double ttm_peak(const orc_sys *S, double P0)
{
    double *Te = malloc(sizeof(double) * S->nc), *Tl = malloc(sizeof(double) * S->nc);
    for (int c = 0; c < S->nc; ++c) { Te[c] = S->t.T0; Tl[c] = S->t.T0; }
    double sig = pulse_sigma(&S->t), t0 = pulse_t0(&S->t);
    double tend = t0 + 10.0 * sig;
    double Dt = ttm_dt(S);
    int64_t nsteps = (int64_t)ceil(tend / Dt);
    double peak = S->t.T0;
    for (int64_t n = 0; n < nsteps; ++n) {
        ttm_advance(S, Te, Tl, n * Dt, Dt, P0, 1);
        for (int c = 0; c < S->nc; ++c) if (Te[c] > peak) peak = Te[c];
    }
    free(Te); free(Tl);
    return peak;
}

int orc_set_ttm(orc_sys *S, const orc_ttm *t, char *err, int errlen)
{
    if (!S->periodic) { snprintf(err, errlen, "TTM grid needs a periodic lattice"); return -1; }
    if (t->ncx < 1 || t->ncy < 1 || t->ncz < 1) { snprintf(err, errlen, "bad TTM grid"); return -1; }
    S->t = *t;
    S->has_ttm = 1;
    S->nc = t->ncx * t->ncy * t->ncz;
    free(S->Te); free(S->Tl); free(S->cell_of); free(S->src_shape); free(S->scratch);
    S->Te = malloc(sizeof(double) * S->nc);
    S->scratch = malloc(sizeof(double) * 2 * S->nc);
    S->Tl = malloc(sizeof(double) * S->nc);
    S->src_shape = malloc(sizeof(double) * S->nc);
    S->cell_of = malloc(sizeof(int) * S->n);
    int nd[3] = {t->ncx, t->ncy, t->ncz};
    int nl[3] = {S->p.nx, S->p.ny, S->p.nz};
    for (int d = 0; d < 3; ++d) S->dxc[d] = S->box[d] * ANG / nd[d];
    S->cellvol = S->dxc[0] * S->dxc[1] * S->dxc[2];
    for (int c = 0; c < S->nc; ++c) {
        S->Te[c] = t->source == 3 ? profile_Te(t, S->step * ttm_dt(S)) : t->T0;
        S->Tl[c] = t->T0;
    }
    /* cell of atom: floor(x / L * n) evaluated exactly on the half-lattice
     * integer coordinate, so atoms on a cell face go to the upper cell */
    for (int i = 0; i < S->n; ++i) {
        int cc[3];
        for (int d = 0; d < 3; ++d) cc[d] = (int)(((long)S->ipos2[3 * i + d] * nd[d]) / (2L * nl[d]));
        S->cell_of[i] = (cc[2] * t->ncy + cc[1]) * t->ncx + cc[0];
    }
    for (int cz = 0; cz < t->ncz; ++cz)
        for (int cy = 0; cy < t->ncy; ++cy)
            for (int cx = 0; cx < t->ncx; ++cx) {
                int c = (cz * t->ncy + cy) * t->ncx + cx;
                double x = (cx + 0.5) * S->box[0] / t->ncx, y = (cy + 0.5) * S->box[1] / t->ncy;
                double z = (cz + 0.5) * S->box[2] / t->ncz;
                /* laser spot (Sec. II.B source): a Gaussian of width sigma_xy
                 * centred on the box in x-y, or an exponential absorption
                 * profile exp(-z / depth) from the z = 0 face, at cell centres.
                 * The ORC_PLANT_* switches build deliberately wrong variants
                 * for the tests that show the source pins catch such errors;
                 * the normal build defines none of them. */
                double xc = 0.5 * S->box[0], yc = 0.5 * S->box[1], w2 = 2.0 * sq(t->sigma_xy), zs = -1.0;
#ifdef ORC_PLANT_SPOT_NO_HALF
                w2 = sq(t->sigma_xy);
#endif
#ifdef ORC_PLANT_SPOT_OFF_CENTRE
                xc += 0.5 * S->box[0] / t->ncx;
#endif
#ifdef ORC_PLANT_DEPTH_SIGN
                zs = 1.0;
#endif
                double f = 1.0;
                if (t->spatial == 1)
                    f = exp(-(sq(x - xc) + sq(y - yc)) / w2);
                else if (t->spatial == 2)
                    f = exp(zs * z / t->depth_z);
                S->src_shape[c] = f;
            }
    /* sub-steps: smallest m with dt/m <= 0.4 C_e(T0) dx_min^2 / (kappa_e d) */
    int d = 0;
    double dxmin = 1e300;
    for (int k = 0; k < 3; ++k) if (nd[k] > 1) { ++d; if (S->dxc[k] < dxmin) dxmin = S->dxc[k]; }
    S->substeps = 1;
    if (d > 0 && t->kappa_e > 0.0 && t->source != 3) {
        double dmax = 0.4 * t->gamma_e * t->T0 * dxmin * dxmin / (t->kappa_e * d);
        double m = ceil(ttm_dt(S) / dmax);
        S->substeps = m < 1.0 ? 1 : (int)m;
    }
    S->P0 = t->P0;
    if (t->source == 1) {
        /* bisection on P0 so that the peak of T_e over cells and steps is peak_Te */
        double target = t->peak_Te;
        double sig = pulse_sigma(t);
        double Eneed = 0.5 * t->gamma_e * (target * target - t->T0 * t->T0);
        double hi = Eneed / (sig * sqrt(2.0 * PI));
        while (ttm_peak(S, hi) < target) hi *= 2.0;
        double lo = 0.0;
        for (int it = 0; it < 60; ++it) {
            double mid = 0.5 * (lo + hi);
            if (ttm_peak(S, mid) < target) lo = mid; else hi = mid;
        }
        S->P0 = 0.5 * (lo + hi);
    }
    S->src_energy = 0.0;
    if (S->lattice_on) rebuild_lists(S);   /* bath cells from the current positions */
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Field, noise and the symmetric sweep                                      */
/* ------------------------------------------------------------------------- */

/* Deterministic field in tesla, B_i = (1/mu_i)[sum_j J_ij s_j + 2 K (s_i.n) n] + B_ext. */
void orc_field(const orc_sys *S, int i, double Bo[3])
{
    double h[3] = {0, 0, 0};
    for (int k = S->nbr_start[i]; k < S->nbr_start[i + 1]; ++k) {
        int j = S->nbr_j[k];
        double J = S->nbr_J[k];
        h[0] += J * S->s[3 * j];
        h[1] += J * S->s[3 * j + 1];
        h[2] += J * S->s[3 * j + 2];
    }
    int t = S->species[i];
    const double *n = S->p.axis;
    double sn = S->s[3 * i] * n[0] + S->s[3 * i + 1] * n[1] + S->s[3 * i + 2] * n[2];
    double mu = S->p.mu[t] * MUB;
    for (int k = 0; k < 3; ++k)
        Bo[k] = (h[k] + 2.0 * S->p.K[t] * sn * n[k]) / mu + S->p.B[k];
}

static double bath_T(const orc_sys *S, int i)
{
    return S->has_ttm ? S->Te[S->cell_of[i]] : S->p.T_bath;
}

/* Noise amplitude for a sub-step of length h: sqrt(2 alpha k_B T / (gamma mu h)),
 * the FDT value whose 1/sqrt(mu) scaling is the mu_fdt option of Sec. II.C.
 * A test may set noise_mu_power = 1 to reproduce the variant without mu_fdt,
 * in which the torque rescaling mu_ref/mu also multiplies the noise, i.e. an
 * extra factor sqrt(mu_ref/mu) with mu_ref the moment of species 0. */
static double noise_sigma(const orc_sys *S, int t, double T, double h)
{
    double mu = S->p.mu[t] * MUB;
    double a = S->p.alpha[t];
    double fdt = sqrt(2.0 * a * KB * T / (GAMMA * mu * h));
    return fdt * pow(S->p.mu[0] / S->p.mu[t], S->p.noise_mu_power - 0.5);
}

/* Field used for one sub-step of atom i.  The exchange, Zeeman and noise parts
 * do not depend on s_i and are held fixed over the sub-step; the on-site
 * anisotropy part kappa (s.n) n, kappa = 2K/mu, does, so it is taken at the
 * sub-step midpoint predicted from the rate of change of c = s.n under Eq. 1:
 *   dc/dt = -gamma' [ n.(s x B) + alpha ( c (s.B) - n.B ) ],
 *   B_sub = B + kappa (h/2) (dc/dt) n,
 * which makes the single-spin sub-step accurate to O(h^3) locally, so the
 * symmetric sweep stays second order when anisotropy is present. */
static void substep_field(const orc_sys *S, int i, const double B[3], double h, double out[3])
{
    int t = S->species[i];
    const double *n = S->p.axis;
    const double *s = &S->s[3 * i];
    double kappa = 2.0 * S->p.K[t] / (S->p.mu[t] * MUB);
    double a = S->p.alpha[t];
    double gp = GAMMA / (1.0 + a * a);
    double c = s[0] * n[0] + s[1] * n[1] + s[2] * n[2];
    double sxB[3] = {s[1] * B[2] - s[2] * B[1], s[2] * B[0] - s[0] * B[2], s[0] * B[1] - s[1] * B[0]};
    double n_sxB = n[0] * sxB[0] + n[1] * sxB[1] + n[2] * sxB[2];
    double sB = s[0] * B[0] + s[1] * B[1] + s[2] * B[2];
    double nB = n[0] * B[0] + n[1] * B[1] + n[2] * B[2];
    double cdot = -gp * (n_sxB + a * (c * sB - nB));
    for (int k = 0; k < 3; ++k) out[k] = B[k] + kappa * 0.5 * h * cdot * n[k];
}

/* One colour pass: every atom of colour c advanced by h, pass index p. */
static void colour_pass(orc_sys *S, int c, double h, uint32_t pass)
{
    uint32_t key[2] = {(uint32_t)(S->p.seed & 0xffffffffu), (uint32_t)(S->p.seed >> 32)};
    for (int i = 0; i < S->n; ++i) {
        if (S->colour[i] != c) continue;
        double B[3], Bs[3];
        orc_field(S, i, B);
        int t = S->species[i];
        double T = bath_T(S, i);
        if (T > 0.0 && S->p.alpha[t] > 0.0) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)S->step, pass, S->p.instance}, w[4];
            double g[3];
            orc_philox4x32_10(ctr, key, w);
            orc_gauss3(w, g);
            double sg = noise_sigma(S, t, T, h);
            for (int k = 0; k < 3; ++k) B[k] += sg * g[k];
        }
        substep_field(S, i, B, h, Bs);
        orc_flow(&S->s[3 * i], Bs, S->p.alpha[t], h);
    }
}

static void record_sample(orc_sys *S)
{
    if (S->nsamp == S->capsamp) {
        S->capsamp = S->capsamp ? 2 * S->capsamp : 64;
        S->samples = realloc(S->samples, sizeof(double) * ORC_NOBS * S->capsamp);
    }
    orc_observe(S, &S->samples[ORC_NOBS * S->nsamp]);
    S->nsamp++;
}

/* One step t_n -> t_n+1: the bath reads T_e(t_n); passes p = 0..K-2 take
 * colours 0..K-2 with h = dt/2, pass K-1 takes colour K-1 with h = dt, passes
 * K..2K-2 take colours K-2..0 with h = dt/2; then the TTM grid advances. */
static void spin_sweep(orc_sys *S)
{
    int K = S->ncolours;
    double dt = S->p.dt;
    uint32_t pass = 0;
    for (int c = 0; c < K - 1; ++c) colour_pass(S, c, 0.5 * dt, pass++);
    colour_pass(S, K - 1, dt, pass++);
    for (int c = K - 2; c >= 0; --c) colour_pass(S, c, 0.5 * dt, pass++);
}

/* Merged sweep, one step (K >= 2).  The leading pass of colour 0 is A_0(dt/2)
 * when the previous step closed, else the bridge A_0(dt) that merges the
 * previous step's trailing half with this step's leading half; it is centred
 * on t_n, so it uses this step's bath T_e(t_n), counter (atom, n, pass 0) and
 * the full-step noise amplitude.  Inner passes as in the symmetric sweep; the
 * trailing A_0(dt/2) (pass 2K-2) only when the step closes. */
static void merged_sweep(orc_sys *S, int open, int close)
{
    int K = S->ncolours;
    double dt = S->p.dt;
    uint32_t pass = 0;
    colour_pass(S, 0, open ? dt : 0.5 * dt, pass++);
    for (int c = 1; c < K - 1; ++c) colour_pass(S, c, 0.5 * dt, pass++);
    colour_pass(S, K - 1, dt, pass++);
    for (int c = K - 2; c >= 1; --c) colour_pass(S, c, 0.5 * dt, pass++);
    if (close) colour_pass(S, 0, 0.5 * dt, pass);
}

void orc_step(orc_sys *S, int64_t nsteps)
{
    double dt = S->p.dt;
    int merged = S->p.sweep == 1 && S->ncolours >= 2;
    int open = 0;
    for (int64_t it = 0; it < nsteps; ++it) {
        if (merged) {
            int sample = S->p.sample_every > 0 && (S->step + 1) % S->p.sample_every == 0;
            int close = sample || it == nsteps - 1;
            merged_sweep(S, open, close);
            open = !close;
        } else {
            spin_sweep(S);
        }
        if (S->has_ttm)
            S->src_energy += ttm_advance(S, S->Te, S->Tl, S->step * dt, dt, S->P0, 1);
        S->step++;
        if (S->p.sample_every > 0 && S->step % S->p.sample_every == 0) record_sample(S);
    }
}

/* Observable record (all double):
 *  [0] t  [1..3] mean s of species 0  [4..6] mean s of species 1
 *  [7..9] moment-weighted net direction sum(mu_i s_i) / sum(mu_i)
 *  [10] exchange energy -sum_{i<j} J_ij s_i.s_j  [11] anisotropy -sum K (s.n)^2
 *  [12] Zeeman -sum mu_i B.s_i  [13..14] spin temperature per species
 *  sum |s x H|^2 / (2 k_B sum s.H), H = mu_i B_i (deterministic)
 *  [15] mean T_e  [16] mean T_l  [17] lattice kinetic energy  [18] lattice
 *  potential energy  [19] step count. */
void orc_observe(const orc_sys *S, double o[ORC_NOBS])
{
    memset(o, 0, sizeof(double) * ORC_NOBS);
    o[0] = S->step * S->p.dt;
    double cnt[2] = {0, 0}, num[2] = {0, 0}, den[2] = {0, 0}, musum = 0.0;
    double Eex = 0.0, Ean = 0.0, EZ = 0.0;
    const double *n = S->p.axis;
    for (int i = 0; i < S->n; ++i) {
        int t = S->species[i];
        const double *si = &S->s[3 * i];
        double mu = S->p.mu[t] * MUB;
        for (int k = 0; k < 3; ++k) { o[1 + 3 * t + k] += si[k]; o[7 + k] += S->p.mu[t] * si[k]; }
        musum += S->p.mu[t];
        cnt[t] += 1.0;
        for (int k = S->nbr_start[i]; k < S->nbr_start[i + 1]; ++k) {
            int j = S->nbr_j[k];
            if (j <= i) continue;
            const double *sj = &S->s[3 * j];
            Eex -= S->nbr_J[k] * (si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2]);
        }
        double sn = si[0] * n[0] + si[1] * n[1] + si[2] * n[2];
        Ean -= S->p.K[t] * sn * sn;
        EZ -= mu * (S->p.B[0] * si[0] + S->p.B[1] * si[1] + S->p.B[2] * si[2]);
        double B[3], H[3];
        orc_field(S, i, B);
        for (int k = 0; k < 3; ++k) H[k] = mu * B[k];
        double cx = si[1] * H[2] - si[2] * H[1];
        double cy = si[2] * H[0] - si[0] * H[2];
        double cz = si[0] * H[1] - si[1] * H[0];
        num[t] += cx * cx + cy * cy + cz * cz;
        den[t] += si[0] * H[0] + si[1] * H[1] + si[2] * H[2];
    }
    for (int t = 0; t < 2; ++t) {
        if (cnt[t] > 0) for (int k = 0; k < 3; ++k) o[1 + 3 * t + k] /= cnt[t];
        o[13 + t] = (cnt[t] > 0 && den[t] != 0.0) ? num[t] / (2.0 * KB * den[t]) : 0.0;
    }
    for (int k = 0; k < 3; ++k) o[7 + k] /= musum;
    o[10] = Eex; o[11] = Ean; o[12] = EZ;
    if (S->has_ttm) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < S->nc; ++c) { a += S->Te[c]; b += S->Tl[c]; }
        o[15] = a / S->nc; o[16] = b / S->nc;
    } else {
        o[15] = S->p.T_bath; o[16] = S->p.T_bath;
    }
    if (S->lattice_on) {
        double ek, em;
        orc_lattice_energy(S, &ek, &em);
        o[16] = 2.0 * ek / (3.0 * S->n * KB);   /* ion kinetic temperature */
        o[17] = ek;
        o[18] = em;
    }
    o[19] = (double)S->step;
}

/* ------------------------------------------------------------------------- */
/* Accessors                                                                 */
/* ------------------------------------------------------------------------- */
int orc_natoms(const orc_sys *S) { return S->n; }
int orc_ncolours(const orc_sys *S) { return S->ncolours; }
int64_t orc_stepcount(const orc_sys *S) { return S->step; }
void orc_set_stepcount(orc_sys *S, int64_t n) { S->step = n; }
void orc_get_spins(const orc_sys *S, double *out) { memcpy(out, S->s, sizeof(double) * 3 * S->n); }
void orc_set_spins(orc_sys *S, const double *in) { memcpy(S->s, in, sizeof(double) * 3 * S->n); }
void orc_get_species(const orc_sys *S, int *out) { memcpy(out, S->species, sizeof(int) * S->n); }
void orc_get_colours(const orc_sys *S, int *out) { memcpy(out, S->colour, sizeof(int) * S->n); }
void orc_get_positions(const orc_sys *S, double *out) { memcpy(out, S->pos, sizeof(double) * 3 * S->n); }
int orc_neighbour_count(const orc_sys *S, int i) { return S->nbr_start[i + 1] - S->nbr_start[i]; }
void orc_get_neighbours(const orc_sys *S, int i, int *j_out, double *J_out)
{
    int c = 0;
    for (int k = S->nbr_start[i]; k < S->nbr_start[i + 1]; ++k, ++c) {
        j_out[c] = S->nbr_j[k];
        J_out[c] = S->nbr_J[k];
    }
}
int64_t orc_nsamples(const orc_sys *S) { return S->nsamp; }
void orc_get_samples(const orc_sys *S, double *out)
{
    if (S->nsamp) memcpy(out, S->samples, sizeof(double) * ORC_NOBS * S->nsamp);
}
double orc_ttm_P0(const orc_sys *S) { return S->P0; }
int orc_ttm_substeps(const orc_sys *S) { return S->substeps; }
int orc_ttm_ncells(const orc_sys *S) { return S->has_ttm ? S->nc : 0; }
void orc_ttm_get(const orc_sys *S, double *Te, double *Tl)
{
    memcpy(Te, S->Te, sizeof(double) * S->nc);
    memcpy(Tl, S->Tl, sizeof(double) * S->nc);
}
void orc_ttm_set(orc_sys *S, const double *Te, const double *Tl)
{
    memcpy(S->Te, Te, sizeof(double) * S->nc);
    memcpy(S->Tl, Tl, sizeof(double) * S->nc);
}
double orc_ttm_source_energy(const orc_sys *S) { return S->src_energy; }
int orc_atom_cell(const orc_sys *S, int i) { return S->has_ttm ? S->cell_of[i] : 0; }

/* ------------------------------------------------------------------------- */
/* Moving lattice                                                            */
/*                                                                           */
/* One lattice step of length dtL = m dt (m = spin_substeps):                */
/*   v += F dtL / 2M; m/2 spin steps; x += v dtL; new pair lists and J(r_ij);*/
/*   m/2 spin steps; F = F_Morse + F_mag; v += F dtL / 2M;                   */
/*   electron-ion coupling: v <- c1 v + c2 xi with c1 = exp(-gamma dtL / M), */
/*   c2 = sqrt(k_B T_e (1 - c1^2) / M), the exact Ornstein-Uhlenbeck update  */
/*   of the friction + noise force -gamma v + sqrt(2 gamma k_B T_e) xi(t),   */
/*   whose kinetic-energy change is taken from the electrons of the atom's   */
/*   TTM cell; then the TTM grid advances over dtL without its G term.       */
/* F_mag,i = -sum_j J'(r_ij) (s_i.s_j) rhat_ij with rhat_ij from i to j, the  */
/* exchange-mediated force of Sec. II.A; F_Morse,i = sum_j U'(r_ij) rhat_ij. */
/* ------------------------------------------------------------------------- */
/* Morse pair energy D [e^{-2a(r-r0)} - 2 e^{-a(r-r0)}] and its derivative */
static double morse_raw(const orc_lattice *L, double r)
{
    double e1 = exp(-L->morse_alpha * (r - L->morse_r0));
    return L->morse_D * (e1 * e1 - 2.0 * e1);
}

static double morse_raw_dU(const orc_lattice *L, double r)   /* J per angstrom */
{
    double e1 = exp(-L->morse_alpha * (r - L->morse_r0));
    return 2.0 * L->morse_alpha * L->morse_D * (e1 - e1 * e1);
}

/* shifted-force form: energy and force both vanish at the cutoff,
 * U_sf(r) = U(r) - U(rc) - (r - rc) U'(rc) */
static double morse_U(const orc_lattice *L, double r)
{
    double rc = L->morse_rc;
    return morse_raw(L, r) - morse_raw(L, rc) - (r - rc) * morse_raw_dU(L, rc);
}

static double morse_dU(const orc_lattice *L, double r)
{
    return morse_raw_dU(L, r) - morse_raw_dU(L, L->morse_rc);
}

static double pair_dJ(const orc_params *p, int ti, int tj, double r)   /* J per angstrom */
{
    const orc_exch *e = &p->exch[ti][tj];
    if (e->kind != 2 || r >= e->rc) return 0.0;
    return orc_bethe_slater_deriv(r, e->J1, e->J2, e->J3);
}

static void wrap_positions(orc_sys *S)
{
    for (int i = 0; i < S->n; ++i)
        for (int k = 0; k < 3; ++k) {
            double L = S->box[k];
            double x = S->pos[3 * i + k];
            x -= L * floor(x / L);
            if (x >= L) x -= L;
            S->pos[3 * i + k] = x;
        }
}

static int finite_pos(const orc_sys *S, int i)
{
    return isfinite(S->pos[3 * i]) && isfinite(S->pos[3 * i + 1]) && isfinite(S->pos[3 * i + 2]);
}

/* all j != i with minimum-image distance below rc, ascending j, as CSR; cell
 * list with cells no smaller than rc (brute force when fewer than 3 cells).
 * Atoms whose position is not finite (a run that has blown up) take part in
 * no pair, so that the state stays inspectable instead of every pair
 * qualifying. */
static void pairs_within(const orc_sys *S, double rc, int **pstart, int **pj)
{
    int n = S->n;
    int nc[3], brute = 0;
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(S->box[k] / rc);
        if (nc[k] < 3) brute = 1;
    }
    int *start = malloc(sizeof(int) * (n + 1));
    int cap = n * 16 + 16, total = 0;
    int *jl = malloc(sizeof(int) * cap);
    int *head = NULL, *next = NULL, *cellof = NULL;
    if (!brute) {
        head = malloc(sizeof(int) * nc[0] * nc[1] * nc[2]);
        next = malloc(sizeof(int) * n);
        cellof = malloc(sizeof(int) * n * 3);
        for (int c = 0; c < nc[0] * nc[1] * nc[2]; ++c) head[c] = -1;
        for (int i = n - 1; i >= 0; --i) {
            int cc[3];
            if (!finite_pos(S, i)) { next[i] = -1; cellof[3 * i] = -1; continue; }
            for (int k = 0; k < 3; ++k) {
                cc[k] = (int)floor(S->pos[3 * i + k] / S->box[k] * nc[k]);
                if (cc[k] >= nc[k]) cc[k] = nc[k] - 1;
                if (cc[k] < 0) cc[k] = 0;
                cellof[3 * i + k] = cc[k];
            }
            int c = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
            next[i] = head[c];
            head[c] = i;
        }
    }
    int tcap = 64, *tmp = malloc(sizeof(int) * tcap);
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        if (!finite_pos(S, i)) {
            /* an atom whose position is not finite has no neighbours */
        } else if (brute) {
            for (int j = 0; j < n; ++j) {
                if (j == i || !finite_pos(S, j)) continue;
                double d[3];
                min_image(S, i, j, d);
                if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) >= rc) continue;
                if (cnt == tcap) { tcap *= 2; tmp = realloc(tmp, sizeof(int) * tcap); }
                tmp[cnt++] = j;
            }
        } else {
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int cx = (cellof[3 * i] + dx + nc[0]) % nc[0];
                        int cy = (cellof[3 * i + 1] + dy + nc[1]) % nc[1];
                        int cz = (cellof[3 * i + 2] + dz + nc[2]) % nc[2];
                        for (int j = head[(cz * nc[1] + cy) * nc[0] + cx]; j >= 0; j = next[j]) {
                            if (j == i) continue;
                            double d[3];
                            min_image(S, i, j, d);
                            if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) >= rc) continue;
                            if (cnt == tcap) { tcap *= 2; tmp = realloc(tmp, sizeof(int) * tcap); }
                            tmp[cnt++] = j;
                        }
                    }
        }
        qsort(tmp, cnt, sizeof(int), cmp_int);
        start[i] = total;
        for (int k = 0; k < cnt; ++k) {
            if (total == cap) { cap *= 2; jl = realloc(jl, sizeof(int) * cap); }
            jl[total++] = tmp[k];
        }
    }
    start[n] = total;
    free(tmp); free(head); free(next); free(cellof);
    *pstart = start;
    *pj = jl;
}

/* exchange list with J(r) at the current positions, Morse list, colour check */
static void rebuild_lists(orc_sys *S)
{
    int *st, *jj;
    pairs_within(S, max_rc(&S->p), &st, &jj);
    free(S->nbr_start); free(S->nbr_j); free(S->nbr_J);
    S->nbr_start = malloc(sizeof(int) * (S->n + 1));
    S->nbr_j = malloc(sizeof(int) * (st[S->n] + 1));
    S->nbr_J = malloc(sizeof(double) * (st[S->n] + 1));
    int total = 0;
    S->colour_violations = 0;
    for (int i = 0; i < S->n; ++i) {
        S->nbr_start[i] = total;
        for (int k = st[i]; k < st[i + 1]; ++k) {
            int j = jj[k];
            double d[3];
            min_image(S, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double J = pair_J(&S->p, S->species[i], S->species[j], r);
            if (J == 0.0) continue;
            if (S->colour[i] == S->colour[j]) S->colour_violations++;
            S->nbr_j[total] = j;
            S->nbr_J[total] = J;
            ++total;
        }
    }
    S->nbr_start[S->n] = total;
    free(st); free(jj);
    free(S->mor_start); free(S->mor_j);
    pairs_within(S, S->L.morse_rc, &S->mor_start, &S->mor_j);
    /* bath cell of each atom from its current position */
    if (S->has_ttm) {
        int nd[3] = {S->t.ncx, S->t.ncy, S->t.ncz};
        for (int i = 0; i < S->n; ++i) {
            int cc[3];
            for (int d = 0; d < 3; ++d) {
                double f = S->pos[3 * i + d] / S->box[d];
                cc[d] = (int)floor(f * nd[d]);
                if (cc[d] >= nd[d]) cc[d] = nd[d] - 1;
                if (cc[d] < 0) cc[d] = 0;
            }
            S->cell_of[i] = (cc[2] * nd[1] + cc[1]) * nd[0] + cc[0];
        }
    }
}

static void compute_forces(orc_sys *S)
{
    for (int k = 0; k < 3 * S->n; ++k) S->force[k] = 0.0;
    for (int i = 0; i < S->n; ++i) {
        for (int k = S->mor_start[i]; k < S->mor_start[i + 1]; ++k) {
            int j = S->mor_j[k];
            double d[3];
            min_image(S, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double f = morse_dU(&S->L, r) * 1e10;          /* N */
            for (int c = 0; c < 3; ++c) S->force[3 * i + c] += f * d[c] / r;
        }
        for (int k = S->nbr_start[i]; k < S->nbr_start[i + 1]; ++k) {
            int j = S->nbr_j[k];
            double d[3];
            min_image(S, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double *si = &S->s[3 * i], *sj = &S->s[3 * j];
            double ss = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
            double f = -pair_dJ(&S->p, S->species[i], S->species[j], r) * ss * 1e10;
            for (int c = 0; c < 3; ++c) S->force[3 * i + c] += f * d[c] / r;
        }
    }
}

int orc_set_lattice(orc_sys *S, const orc_lattice *L, char *err, int errlen)
{
    if (!S->periodic) { snprintf(err, errlen, "a moving lattice needs a periodic lattice"); return -1; }
    if (S->has_ttm) { snprintf(err, errlen, "set the moving lattice before the TTM grid"); return -1; }
    if (L->spin_substeps < 2 || L->spin_substeps % 2) { snprintf(err, errlen, "spin_substeps must be even"); return -1; }
    if (!(L->mass_amu > 0.0) || !(L->morse_rc > 0.0)) { snprintf(err, errlen, "bad lattice parameters"); return -1; }
    for (int k = 0; k < 3; ++k)
        if (S->box[k] <= 2.0 * L->morse_rc) { snprintf(err, errlen, "box must exceed twice the pair cutoff"); return -1; }
    S->L = *L;
    S->lattice_on = 1;
    S->mass = L->mass_amu * 1.66053906660e-27;
    S->vel = realloc(S->vel, sizeof(double) * 3 * S->n);
    S->force = realloc(S->force, sizeof(double) * 3 * S->n);
    /* initial longitudinal strain wave along z, one wavelength per box */
    double Lz = S->box[2];
    for (int i = 0; i < S->n; ++i) {
        double z0 = S->pos[3 * i + 2];
        S->pos[3 * i + 2] = z0 + L->strain_amp * Lz / (2.0 * PI) * sin(2.0 * PI * z0 / Lz);
    }
    wrap_positions(S);
    /* Maxwell-Boltzmann velocities (Philox counter (atom, 0, 0xFFFF0003, instance)),
     * net momentum removed */
    uint32_t key[2] = {(uint32_t)(S->p.seed & 0xffffffffu), (uint32_t)(S->p.seed >> 32)};
    double vs = sqrt(KB * L->T_init / S->mass), mean[3] = {0, 0, 0};
    for (int i = 0; i < S->n; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 0xFFFF0003u, S->p.instance}, w[4];
        double g[3];
        orc_philox4x32_10(ctr, key, w);
        orc_gauss3(w, g);
        for (int k = 0; k < 3; ++k) { S->vel[3 * i + k] = vs * g[k]; mean[k] += S->vel[3 * i + k]; }
    }
    for (int i = 0; i < S->n; ++i)
        for (int k = 0; k < 3; ++k) S->vel[3 * i + k] -= mean[k] / S->n;
    S->lstep = 0;
    S->ion_to_e = 0.0;
    rebuild_lists(S);
    compute_forces(S);
    return 0;
}

void orc_lattice_step(orc_sys *S, int64_t nsteps)
{
    int m = S->L.spin_substeps;
    double dtL = m * S->p.dt;
    double M = S->mass;
    uint32_t key[2] = {(uint32_t)(S->p.seed & 0xffffffffu), (uint32_t)(S->p.seed >> 32)};
    double *dEc = S->has_ttm ? calloc(S->nc, sizeof(double)) : NULL;
    for (int64_t it = 0; it < nsteps; ++it) {
        for (int k = 0; k < 3 * S->n; ++k) S->vel[k] += S->force[k] * dtL / (2.0 * M);
        for (int k = 0; k < m / 2; ++k) { spin_sweep(S); S->step++; }
        for (int k = 0; k < 3 * S->n; ++k) S->pos[k] += S->vel[k] * dtL * 1e10;
        wrap_positions(S);
        rebuild_lists(S);
        for (int k = 0; k < m / 2; ++k) { spin_sweep(S); S->step++; }
        compute_forces(S);
        for (int k = 0; k < 3 * S->n; ++k) S->vel[k] += S->force[k] * dtL / (2.0 * M);
        if (S->L.gamma_p > 0.0) {
            double c1 = exp(-S->L.gamma_p * dtL / M);
            if (dEc) for (int c = 0; c < S->nc; ++c) dEc[c] = 0.0;
            for (int i = 0; i < S->n; ++i) {
                double T = bath_T(S, i);
                double c2 = sqrt(KB * T * (1.0 - c1 * c1) / M);
                uint32_t ctr[4] = {(uint32_t)i, (uint32_t)S->lstep, 0xFFFF0002u, S->p.instance}, w[4];
                double g[3], ke0 = 0.0, ke1 = 0.0;
                orc_philox4x32_10(ctr, key, w);
                orc_gauss3(w, g);
                for (int k = 0; k < 3; ++k) {
                    double v0 = S->vel[3 * i + k];
                    double v1 = c1 * v0 + c2 * g[k];
                    ke0 += 0.5 * M * v0 * v0;
                    ke1 += 0.5 * M * v1 * v1;
                    S->vel[3 * i + k] = v1;
                }
                S->ion_to_e -= ke1 - ke0;
                if (dEc) dEc[S->cell_of[i]] -= ke1 - ke0;
            }
            if (dEc)
                for (int c = 0; c < S->nc; ++c) {
                    double Ee = 0.5 * S->t.gamma_e * S->Te[c] * S->Te[c] + dEc[c] / S->cellvol;
                    S->Te[c] = sqrt(2.0 * Ee / S->t.gamma_e);
                }
        }
        if (S->has_ttm)
            S->src_energy += ttm_advance(S, S->Te, S->Tl, S->lstep * dtL, dtL, S->P0, 0);
        S->lstep++;
        if (S->p.sample_every > 0 && S->lstep % S->p.sample_every == 0) record_sample(S);
    }
    free(dEc);
}

int64_t orc_lattice_stepcount(const orc_sys *S) { return S->lstep; }
void orc_get_velocities(const orc_sys *S, double *out) { memcpy(out, S->vel, sizeof(double) * 3 * S->n); }
void orc_set_velocities(orc_sys *S, const double *in) { memcpy(S->vel, in, sizeof(double) * 3 * S->n); }
void orc_set_positions(orc_sys *S, const double *in)
{
    memcpy(S->pos, in, sizeof(double) * 3 * S->n);
    wrap_positions(S);
    if (S->lattice_on) {
        rebuild_lists(S);
        compute_forces(S);
    }
}
void orc_get_forces(const orc_sys *S, double *out) { memcpy(out, S->force, sizeof(double) * 3 * S->n); }
void orc_lattice_energy(const orc_sys *S, double *kin, double *morse)
{
    double ek = 0.0, em = 0.0;
    for (int i = 0; i < S->n; ++i) {
        for (int k = 0; k < 3; ++k) ek += 0.5 * S->mass * S->vel[3 * i + k] * S->vel[3 * i + k];
        for (int k = S->mor_start[i]; k < S->mor_start[i + 1]; ++k) {
            int j = S->mor_j[k];
            if (j <= i) continue;
            double d[3];
            min_image(S, i, j, d);
            em += morse_U(&S->L, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        }
    }
    *kin = ek;
    *morse = em;
}
int orc_colour_violations(const orc_sys *S) { return S->colour_violations; }
double orc_ion_energy_to_electrons(const orc_sys *S) { return S->ion_to_e; }
