/*
 * tts_oracle.h -- interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a slow, literal restatement of the
 * stochastic Landau-Lifshitz-Gilbert spin advance of the three-temperature
 * spin-lattice method (paper Eq. 1, Eq. 2, Sec. II.B, II.C, II.E).  Only the
 * test suite, the package's smoke entry and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Units: SI, except magnetic moments in Bohr magnetons and lengths in angstrom.
 */
#ifndef TTS_ORACLE_H
#define TTS_ORACLE_H

#include <stdint.h>

#define ORC_NOBS 20 /* doubles per observable record, see orc_observe() */

typedef struct {
    int kind;    /* 0 = no coupling, 1 = constant J1 for r < rc, 2 = Bethe-Slater J(r) */
    double J1;   /* J */
    double J2;   /* dimensionless */
    double J3;   /* angstrom */
    double rc;   /* angstrom */
} orc_exch;

typedef struct {
    int lattice;            /* 0 sc, 1 bcc, 2 fcc, 3 explicit open cluster */
    int nx, ny, nz;         /* conventional cells (lattice 0..2) */
    double a;               /* lattice constant, angstrom */
    int n_explicit;         /* lattice 3: number of atoms */
    const double *pos_explicit;      /* lattice 3: 3*n positions, angstrom */
    const int *species_explicit;     /* lattice 3: species per atom */
    int nspecies;           /* 1 or 2 */
    double mu[2];           /* moments, Bohr magnetons */
    double frac1;           /* fraction of sites holding species 1 (lattices 0..2) */
    orc_exch exch[2][2];    /* exchange model per species pair (symmetric) */
    double K[2];            /* uniaxial anisotropy energy per atom, J */
    double axis[3];         /* anisotropy axis (unit) */
    double B[3];            /* applied field, T */
    double alpha[2];        /* Gilbert damping per species */
    double dt;              /* spin time step, s */
    double T_bath;          /* bath temperature used while no TTM grid is set, K */
    double init_dir[2][3];  /* initial spin direction per species (normalised here) */
    uint64_t seed;          /* Philox key */
    uint32_t instance;      /* realisation / instance id (Philox counter word 3) */
    int sample_every;       /* record observables every this many steps (0 = never) */
    double noise_mu_power;  /* 0.5: FDT noise ~ mu^-1/2; 1: the variant without mu_fdt */
    int sweep;              /* 0 symmetric sweep per step; 1 merged sweep (see orc_step) */
    double colour_rc;       /* 0, or a distance (angstrom) above the exchange cutoff within
                               which no two atoms share a colour */
} orc_params;

typedef struct {
    int ncx, ncy, ncz;      /* grid cells */
    double gamma_e;         /* C_e = gamma_e * T_e, J m^-3 K^-2 */
    double C_l;             /* lattice heat capacity, J m^-3 K^-1 */
    double G;               /* electron-phonon coupling, W m^-3 K^-1 */
    double kappa_e;         /* electron conductivity, W m^-1 K^-1 */
    double T0;              /* initial T_e = T_l, K */
    int source;             /* 0 none, 1 calibrate P0 to peak_Te, 2 fixed P0, 3 step profile:
                               T_e = peak_Te for t < t0, peak_Te / 2 for t0 <= t < t0 + fwhm,
                               T0 after; T_l = T0 (prescribed, no grid equation) */
    double peak_Te;         /* K */
    double P0;              /* W m^-3 */
    double fwhm;            /* s */
    double t0;              /* pulse centre, s; negative selects 3 sigma_t */
    int spatial;            /* 0 uniform, 1 Gaussian spot in x-y, 2 exponential in z */
    double sigma_xy;        /* angstrom */
    double depth_z;         /* angstrom */
} orc_ttm;

/* Moving lattice (paper Sec. II.A: positions under the pair potential plus the
 * exchange-mediated force -dJ/dr (s_i.s_j), advanced together with the spins). */
typedef struct {
    double mass_amu;      /* atomic mass */
    double morse_D;       /* J */
    double morse_alpha;   /* 1/angstrom */
    double morse_r0;      /* angstrom */
    double morse_rc;      /* angstrom; the energy is shifted to zero there */
    int spin_substeps;    /* spin steps per lattice step (even, >= 2) */
    double strain_amp;    /* initial u_z = A Lz / (2 pi) sin(2 pi z / Lz) */
    double T_init;        /* initial ion temperature, K */
    double gamma_p;       /* electron-ion friction coefficient, kg/s (0: none) */
} orc_lattice;

typedef struct orc_sys orc_sys;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in (0,1) from one 32-bit word: ((x >> 9) + 0.5) * 2^-23. */
double orc_uniform(uint32_t x);
/* Three standard normals from one Philox block (Box-Muller). */
void orc_gauss3(const uint32_t w[4], double g[3]);

/* Bethe-Slater radial exchange and its derivative (Sec. II.E). r in angstrom. */
double orc_bethe_slater(double r, double J1, double J2, double J3);
double orc_bethe_slater_deriv(double r, double J1, double J2, double J3);
/* Re-derivation of (J2, J3) that puts the extremum at r1 (Sec. II.E). */
int orc_rederive_exchange(double r1, double *x1, double *J2, double *J3);

/* One sub-step of the single-spin exact frozen-field flow.  s, Bfield (T) in,
 * s updated in place.  Exposed for closed-form tests. */
void orc_flow(double s[3], const double Bfield[3], double alpha, double h);

orc_sys *orc_create(const orc_params *p, char *err, int errlen);
void orc_free(orc_sys *s);
int orc_set_ttm(orc_sys *s, const orc_ttm *t, char *err, int errlen);
/* Advance nsteps spin steps.  Symmetric sweep (sweep = 0): every step is
 * A_0(dt/2) .. A_{K-2}(dt/2) A_{K-1}(dt) A_{K-2}(dt/2) .. A_0(dt/2).  Merged
 * sweep (sweep = 1, K >= 2): the trailing A_0(dt/2) of a step and the leading
 * A_0(dt/2) of the next are one pass A_0(dt) centred on the step boundary; the
 * sweep closes with A_0(dt/2) at every sampling step and at the end of the
 * call, so observables and the state between calls are at whole steps. */
void orc_step(orc_sys *s, int64_t nsteps);

int orc_natoms(const orc_sys *s);
int orc_ncolours(const orc_sys *s);
int64_t orc_stepcount(const orc_sys *s);
void orc_set_stepcount(orc_sys *s, int64_t n);
void orc_get_spins(const orc_sys *s, double *out);
void orc_set_spins(orc_sys *s, const double *in);
void orc_get_species(const orc_sys *s, int *out);
void orc_get_colours(const orc_sys *s, int *out);
void orc_get_positions(const orc_sys *s, double *out);
int orc_neighbour_count(const orc_sys *s, int i);
void orc_get_neighbours(const orc_sys *s, int i, int *j_out, double *J_out);
void orc_field(const orc_sys *s, int i, double B_out[3]);
void orc_observe(const orc_sys *s, double out[ORC_NOBS]);
int64_t orc_nsamples(const orc_sys *s);
void orc_get_samples(const orc_sys *s, double *out);
double orc_ttm_P0(const orc_sys *s);
int orc_ttm_substeps(const orc_sys *s);
int orc_ttm_ncells(const orc_sys *s);
void orc_ttm_get(const orc_sys *s, double *Te, double *Tl);
void orc_ttm_set(orc_sys *s, const double *Te, const double *Tl);
double orc_ttm_source_energy(const orc_sys *s);
int orc_atom_cell(const orc_sys *s, int i);

int orc_set_lattice(orc_sys *s, const orc_lattice *L, char *err, int errlen);
void orc_lattice_step(orc_sys *s, int64_t nsteps);
int64_t orc_lattice_stepcount(const orc_sys *s);
void orc_get_velocities(const orc_sys *s, double *out);   /* m/s */
void orc_set_positions(orc_sys *s, const double *in);     /* angstrom; rebuilds lists and forces */
void orc_set_velocities(orc_sys *s, const double *in);
void orc_get_forces(const orc_sys *s, double *out);       /* N, Morse + magnetic */
/* kinetic and pair-potential energies (J) */
void orc_lattice_energy(const orc_sys *s, double *kinetic, double *morse);
int orc_colour_violations(const orc_sys *s);
double orc_ion_energy_to_electrons(const orc_sys *s);

#endif
