/*
 * tts.h -- C ABI of the B300 (sm_103a) stochastic spin-dynamics library.
 *
 * The library advances classical atomic spins under the stochastic
 * Landau-Lifshitz-Gilbert equation (paper Eq. 1) with a Langevin bath whose
 * temperature is the local electron temperature of a two-temperature-model
 * grid (paper Eq. 2, Sec. II.B, "fix langevin/spin/ttm"), deterministic
 * torques scaled by 1/mu_i and noise scaled by 1/sqrt(mu_i) (Sec. II.C,
 * "fix moment/scale/spin" with "mu_fdt"), exchange from a constant or
 * Bethe-Slater radial J(r) (Sec. II.E), uniaxial anisotropy and a Zeeman field.
 * The sequential Suzuki-Trotter spin sweep of the paper (Sec. II.A) is done as
 * a graph-coloured symmetric sweep; many independent realisations (the task-
 * level replicas of Sec. II.F) advance together as instances of one system.
 *
 * Conventions
 *  - Units: SI, except moments in Bohr magnetons and lengths in angstrom.
 *  - Every function returns an int status: TTS_OK (0) or a negative TTS_ERR_*.
 *    tts_last_error() returns a message for the calling thread's last failure.
 *    No exception or abort crosses this interface.
 *  - The library owns all device memory of a system.  Host arrays passed in are
 *    read during the call only; host arrays passed out are written during the
 *    call only.
 *  - All work of a system is issued on the CUDA stream given at creation
 *    (a cudaStream_t passed as void*, NULL = legacy default stream).
 *    tts_step() returns once the work is queued; calls that return data to
 *    the host synchronise that stream first.
 *  - Spin arrays at this interface are in canonical atom order: atom id
 *    ((iz * ny + iy) * nx + ix) * nbasis + b for lattices (basis order sc: 0;
 *    bcc: corner, body centre; fcc: (0,0,0), (.5,.5,0), (.5,0,.5), (0,.5,.5)),
 *    and input order for explicit clusters; three doubles (x, y, z) per atom.
 *  - One system handle must not be used from two host threads at once.
 */
#ifndef TTS_H
#define TTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TTS_API __attribute__((visibility("default")))
#else
#define TTS_API
#endif

#define TTS_OK 0
#define TTS_ERR_ARG (-1)            /* invalid argument or descriptor */
#define TTS_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define TTS_ERR_OOM (-3)            /* device or host allocation failed */
#define TTS_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait ran out */
#define TTS_ERR_HEALTH (-5)         /* the device health word flagged a fault */
#define TTS_ERR_STATE (-6)          /* call not valid in the current state */
#define TTS_ERR_UNSUPPORTED (-7)    /* combination not implemented */

#define TTS_MAX_SPECIES 2
#define TTS_NOBS 20

#define TTS_LATTICE_SC 0
#define TTS_LATTICE_BCC 1
#define TTS_LATTICE_FCC 2
#define TTS_LATTICE_CLUSTER 3      /* explicit positions, open boundaries */

#define TTS_EXCH_NONE 0
#define TTS_EXCH_CONST 1           /* J(r) = J1 for r < rc */
#define TTS_EXCH_BETHE_SLATER 2    /* J(r) = 4 J1 x (1 - J2 x) exp(-x), x = (r/J3)^2, r < rc (Sec. II.E) */

#define TTS_ENGINE_AUTO 0          /* pick the fastest engine valid for the system */
#define TTS_ENGINE_GENERAL 1       /* explicit neighbour table, one launch per colour pass */
#define TTS_ENGINE_CHECKER 2       /* sc lattice, even edges: implicit stencil, fused passes */
#define TTS_ENGINE_RESIDENT 3      /* sc lattice: one instance per CTA held in shared memory */

/* Order of the colour passes within and across steps (paper Sec. II.A: the
 * symmetric Suzuki-Trotter splitting over colour classes). */
#define TTS_SWEEP_SYMMETRIC 0      /* every step A_0(dt/2)..A_{K-1}(dt)..A_0(dt/2) */
#define TTS_SWEEP_MERGED 1         /* leapfrog form: the trailing A_0(dt/2) of a step and the
                                      leading A_0(dt/2) of the next run as one A_0(dt) centred
                                      on the step boundary (bath and Philox counter of the new
                                      step); closed with A_0(dt/2) at sampling steps and at the
                                      end of every tts_step call, so observables and the state
                                      seen between calls are at whole steps.  2K-2 passes a
                                      step instead of 2K-1; needs the same colour count K >= 2
                                      in every instance; not with a moving lattice. */

/* Exchange coupling of one species pair.  The pair energy is -J(r) s_i.s_j. */
typedef struct {
    int kind;       /* TTS_EXCH_* */
    double J1;      /* J */
    double J2;      /* dimensionless (Bethe-Slater) */
    double J3;      /* angstrom (Bethe-Slater) */
    double rc;      /* cutoff, angstrom */
} tts_exchange;

/* System description.  Hamiltonian (paper Sec. II.A, II.C):
 *   E = -sum_{i<j} J_ij s_i.s_j - sum_i K_{t_i} (s_i.n)^2 - sum_i mu_i B.s_i
 * and the field of atom i is B_i = -(1/mu_i) dE/ds_i in tesla. */
typedef struct {
    int lattice;                 /* TTS_LATTICE_* */
    int nx, ny, nz;              /* conventional cells of every instance (overridable) */
    double a;                    /* lattice constant, angstrom */
    int n_explicit;              /* cluster: atom count */
    const double *pos_explicit;  /* cluster: 3 * n_explicit positions, angstrom */
    const int *species_explicit; /* cluster: species per atom (NULL = all 0) */
    int nspecies;                /* 1 or 2 */
    double mu_muB[TTS_MAX_SPECIES];   /* moments, Bohr magnetons */
    double frac1;                /* fraction of lattice sites holding species 1 */
    tts_exchange exch[TTS_MAX_SPECIES][TTS_MAX_SPECIES]; /* must be symmetric */
    double K[TTS_MAX_SPECIES];   /* uniaxial anisotropy energy per atom, J */
    double axis[3];              /* anisotropy axis (normalised by the library) */
    double B[3];                 /* applied field, T */
    double alpha[TTS_MAX_SPECIES];    /* Gilbert damping */
    double dt;                   /* time step, s */
    double T_bath;               /* bath temperature while no TTM grid is set, K */
    double init_dir[TTS_MAX_SPECIES][3]; /* initial spin direction per species */
    uint64_t seed;               /* noise and placement key */
    int precision;               /* 32 (float spins) or 64 (double spins) */
    int sample_every;            /* observables every this many steps; 0 = never */
    int obs_capacity;            /* samples kept per instance (ring); 0 = 1024 */
    int n_instances;             /* independent realisations, >= 1 */
    const int *inst_cells;       /* NULL or 3 * n_instances cell counts (lattices) */
    const double *inst_frac1;    /* NULL or n_instances species-1 fractions */
    const double *inst_peak_Te;  /* NULL or n_instances TTM peak temperatures, K */
    const double *inst_fwhm;     /* NULL or n_instances TTM pulse FWHM, s */
    int engine;                  /* TTS_ENGINE_* */
    int instance_base;           /* global id of instance 0 (Philox counter word 3 and
                                    placement stream are keyed by instance_base + index) */
    int sweep;                   /* TTS_SWEEP_* */
    const double *inst_T_bath;   /* NULL or n_instances bath temperatures used while no TTM
                                    grid is set, K (e.g. a temperature scan in one batch) */
    double colour_rc;            /* 0, or a distance (angstrom) above the largest exchange
                                    cutoff: no two atoms closer than it share a colour class
                                    (the lattice rule when it qualifies, else greedy); the
                                    margin a moving lattice needs so that no exchange pair
                                    joins one colour as the atoms move */
} tts_system_desc;

#define TTS_SOURCE_NONE 0
#define TTS_SOURCE_PEAK 1          /* calibrate P0 so that max T_e over cells and steps = peak_Te */
#define TTS_SOURCE_POWER 2         /* use P0 as given */
#define TTS_SOURCE_STEP_PROFILE 3  /* prescribed electron temperature, the three-stage step profile
                                      of the paper's GdFeCo runs (Sec. II.D): T_e = peak_Te for
                                      t < t0, peak_Te / 2 for t0 <= t < t0 + fwhm, T0 after; T_l = T0.
                                      No grid equation (gamma_e, C_l, G, kappa_e unused); peak_Te
                                      and fwhm (the second stage) take the per-instance overrides;
                                      not with a moving lattice. */

#define TTS_SPATIAL_UNIFORM 0
#define TTS_SPATIAL_XY_GAUSS 1     /* exp(-((x-xc)^2 + (y-yc)^2) / (2 sigma_xy^2)) at cell centres */
#define TTS_SPATIAL_Z_EXP 2        /* exp(-z / depth_z) at cell centres */

/* Two-temperature-model grid ("fix ttm" of Sec. II.B), one per instance,
 * periodic, covering the instance's box: explicit update of the electron
 * energy gamma_e T_e^2 / 2 with diffusion kappa_e, exchange G (T_e - T_l) and
 * a source P0 exp(-(t - t0)^2 / (2 sigma_t^2)) f(r), sigma_t = fwhm / (2 sqrt(2 ln 2)). */
typedef struct {
    int cells[3];
    double gamma_e;   /* J m^-3 K^-2 */
    double C_l;       /* J m^-3 K^-1 */
    double G;         /* W m^-3 K^-1 */
    double kappa_e;   /* W m^-1 K^-1 */
    double T0;        /* initial T_e = T_l, K */
    int source;       /* TTS_SOURCE_* */
    double peak_Te;   /* K (per-instance override in the system description) */
    double P0;        /* W m^-3 */
    double fwhm;      /* s (per-instance override in the system description) */
    double t0;        /* pulse centre, s; negative = 3 sigma_t */
    int spatial;      /* TTS_SPATIAL_* */
    double sigma_xy;  /* angstrom */
    double depth_z;   /* angstrom */
} tts_ttm_desc;

typedef struct tts_system tts_system;

/* Moving lattice (paper Sec. II.A): atoms move under a pair potential plus
 * the exchange-mediated force -dJ(r_ij)/dr (s_i.s_j), advanced together with
 * the spins.  One lattice step of length spin_substeps * dt is
 *   v += F dtL/2M; spin_substeps/2 spin steps; x += v dtL; J(r_ij) refreshed;
 *   spin_substeps/2 spin steps; F recomputed; v += F dtL/2M;
 *   electron-ion coupling (exact Ornstein-Uhlenbeck update of the friction
 *   -gamma_p v plus noise at the atom's T_e, the kinetic-energy change taken
 *   from the electrons of its TTM cell); TTM grid advanced by dtL.
 * The pair potential is Morse in shifted-force form (energy and force vanish
 * at morse_rc).  Candidate pairs are those within max(cutoffs) + skin of the
 * reference lattice; an atom that moves further than skin/2 from its site
 * sets the health word (TTS_ERR_HEALTH at tts_sync). */
typedef struct {
    double mass_amu;
    double morse_D;       /* J */
    double morse_alpha;   /* 1/angstrom */
    double morse_r0;      /* angstrom */
    double morse_rc;      /* angstrom */
    int spin_substeps;    /* spin steps per lattice step, even */
    double strain_amp;    /* initial u_z = A Lz / (2 pi) sin(2 pi z / Lz) */
    double T_init;        /* initial ion temperature (Maxwell-Boltzmann, Philox
                             counter (atom, 0, 0xFFFF0003, instance)), K */
    double gamma_p;       /* electron-ion friction, kg/s (0 = none); noise from
                             Philox counter (atom, lattice step, 0xFFFF0002, instance) */
    double skin;          /* angstrom */
} tts_lattice_desc;

/* Facts about a created system. */
typedef struct {
    int64_t n_total;        /* atoms over all instances */
    int n_instances;
    int engine;             /* TTS_ENGINE_* in use */
    int precision;          /* 32 or 64 */
    int max_colours;        /* largest colour count over instances */
    int64_t steps_done;     /* steps completed (device step counter as last synchronised) */
    int64_t kernel_launches;/* kernels this library has launched for the system so far */
} tts_info_t;

/* Build a system: lattice sites, random alloy placement (exactly
 * round(frac1 * N) sites of species 1 per instance, sampled without
 * replacement as in Sec. II.D, drawn from Philox4x32-10 with key = seed and
 * counter (k, attempt, 0xFFFF0000, instance)), neighbour lists, colour
 * classes, device buffers.  Spins start along init_dir of their species and
 * the bath is T_bath until tts_set_ttm_grid().  stream: cudaStream_t or NULL.
 * Errors: TTS_ERR_ARG (bad descriptor, box edge not above twice the cutoff),
 * TTS_ERR_OOM, TTS_ERR_CUDA, TTS_ERR_UNSUPPORTED (engine forced on a system it
 * cannot run).  On error *out is set to NULL. */
TTS_API int tts_create_system(const tts_system_desc *desc, void *stream, tts_system **out);

/* Free all memory of a system (synchronises its stream).  NULL is allowed. */
TTS_API int tts_destroy(tts_system *sys);

/* Attach a TTM grid to every instance (Eq. 2: each atom's bath temperature
 * is T_e of the grid cell that holds it).  Calibrates P0 per instance when
 * source == TTS_SOURCE_PEAK.  Resets T_e = T_l = T0.  Errors: TTS_ERR_ARG,
 * TTS_ERR_UNSUPPORTED (clusters), TTS_ERR_CUDA. */
TTS_API int tts_set_ttm_grid(tts_system *sys, const tts_ttm_desc *ttm);

/* Advance every instance by nsteps time steps (asynchronous).  One step:
 * noise amplitudes from T_e(t_n), the variance 2 alpha k_B T_e / (gamma mu_i h)
 * of the thermal field of the bath coupled to the electron temperature
 * (Eq. 2, Sec. II.B) with the 1/mu_i torque and 1/sqrt(mu_i) noise scaling of
 * Sec. II.C; the stochastic LLG equation (Eq. 1, Sec. II.A) integrated by the
 * symplectic Suzuki-Trotter splitting of Sec. II.A, done as a symmetric sweep
 * over colour classes (each sub-step the exact flow of Eq. 1 under the field
 * held fixed for it); the TTM grid from t_n to t_n+1 (Sec. II.B); observables
 * at t_n+1 when the step count reaches a multiple of sample_every.  Work is
 * queued on the system's stream and nothing is read back.
 * Errors: TTS_ERR_ARG (nsteps < 0), TTS_ERR_CUDA (a launch failed). */
TTS_API int tts_step(tts_system *sys, int64_t nsteps);

/* Wait for queued work and check the device health word.  The paper has no
 * counterpart (its runs are CPU processes): this is the failure check of the
 * device path.  A flagged fault stays flagged for the life of the system
 * (rebuild it, or restore a checkpoint into a new one).  Errors:
 * TTS_ERR_HEALTH (a non-finite spin; with a moving lattice also an atom
 * beyond half its skin, two exchange-coupled atoms of one colour, or a full
 * neighbour table), TTS_ERR_DEVICE_TIMEOUT (a bounded device-side wait ran
 * out; the kernel that waited returned early), TTS_ERR_CUDA. */
TTS_API int tts_sync(tts_system *sys);

/* Bits of the device health word (tts_health).  A kernel that meets one of
 * these conditions sets its bit and goes on (no trap, no abort); tts_sync
 * turns a set word into a status, the bits checked in this order. */
#define TTS_HEALTH_NONFINITE 1u    /* a spin component became NaN or infinite */
#define TTS_HEALTH_TIMEOUT 2u      /* a bounded device-side wait ran out */
#define TTS_HEALTH_SKIN 4u         /* moving lattice: an atom moved beyond half the skin */
#define TTS_HEALTH_COLOUR 8u       /* moving lattice: two exchange-coupled atoms share a colour */
#define TTS_HEALTH_OVERFLOW 16u    /* moving lattice: more exchange neighbours than the table holds */

/* The device health word as it stands (synchronises; TTS_HEALTH_* bits, 0 =
 * no fault).  The paper has no counterpart.  Errors: TTS_ERR_ARG, TTS_ERR_CUDA. */
TTS_API int tts_health(tts_system *sys, unsigned *bits);

/* Self-test of the device's bounded waits, the paper has no counterpart: a
 * one-CTA kernel on the system's stream waits on a shared-memory barrier for
 * a transfer that is never issued, with the library's bounded wait cut to
 * limit_ns; when the wait runs out the kernel sets TTS_HEALTH_TIMEOUT in the
 * system's health word and returns (no trap), so that the next tts_sync
 * reports TTS_ERR_DEVICE_TIMEOUT and the context stays usable.  The flag then
 * stays set like any other fault.  Asynchronous.  Errors: TTS_ERR_ARG
 * (limit_ns outside (0, 10 s]), TTS_ERR_CUDA. */
TTS_API int tts_selftest_wait(tts_system *sys, int64_t limit_ns);

/* Copy up to max_samples observable records of one instance, oldest first,
 * TTS_NOBS doubles each.  These are the quantities the paper follows: the
 * sublattice magnetisations whose z components define switching (Sec. II.G),
 * the energies of the Hamiltonian of Sec. II.A, and the per-sublattice spin
 * temperature of the "compute spin" estimator (Sec. III.A), all reduced in
 * FP64 in a fixed order:
 *  [0] t  [1..3] mean s of species 0  [4..6] mean s of species 1
 *  [7..9] sum(mu_i s_i)/sum(mu_i)  [10] -sum_{i<j} J_ij s_i.s_j
 *  [11] -sum K (s.n)^2  [12] -sum mu_i B.s_i  [13..14] spin temperature per
 *  species, sum|s x H|^2 / (2 k_B sum s.H) with H = mu_i B_i
 *  [15] mean T_e  [16] mean T_l  [17..18] reserved (0)  [19] step count.
 * *n_written receives the count.  Synchronises. */
TTS_API int tts_observables(tts_system *sys, int inst, double *out_host, int64_t max_samples,
                    int64_t *n_written);

/* Record one observable row for an instance now, into out_host (TTS_NOBS
 * doubles), without touching the ring.  Synchronises. */
TTS_API int tts_observe_now(tts_system *sys, int inst, double *out_host);

/* Spins of one instance, 3 doubles per atom, canonical order.  Synchronises. */
TTS_API int tts_get_spins(tts_system *sys, int inst, double *host_xyz);
/* Replace the spins of one instance (normalised by the library). */
TTS_API int tts_set_spins(tts_system *sys, int inst, const double *host_xyz);
/* Spins of all instances, concatenated in instance order (3 doubles each). */
TTS_API int tts_get_all_spins(tts_system *sys, double *host_xyz);
TTS_API int tts_set_all_spins(tts_system *sys, const double *host_xyz);

/* Bulk spin I/O for a host that keeps the state between calls: the spins of
 * all instances, concatenated in instance order and canonical atom order,
 * xyz interleaved, in the system's precision (float for a precision-32
 * system, double for 64); bytes = 3 n_total (4 or 8).  The reordering runs on
 * the device and the copy is one DMA on the system's stream: both calls
 * return once queued, and host_xyz (page-locked memory gives full speed) must
 * stay untouched until the stream reaches the copy (tts_sync).  Written spins
 * are taken as given (not renormalised).  A device staging buffer of the same
 * size is allocated at the first call and kept.
 * Errors: TTS_ERR_ARG (null pointer, wrong byte count), TTS_ERR_OOM,
 * TTS_ERR_CUDA. */
TTS_API int tts_read_spins_async(tts_system *sys, void *host_xyz, size_t bytes);
TTS_API int tts_write_spins_async(tts_system *sys, const void *host_xyz, size_t bytes);

/* Atom count, species (int per atom) and colour class (int per atom) of one
 * instance, canonical order. */
TTS_API int tts_instance_size(tts_system *sys, int inst, int64_t *n_atoms, int *n_colours);
TTS_API int tts_get_species(tts_system *sys, int inst, int *host_species);
TTS_API int tts_get_colours(tts_system *sys, int inst, int *host_colours);

/* T_e, T_l of an instance's grid cells (x fastest) and its source power P0. */
TTS_API int tts_get_ttm(tts_system *sys, int inst, double *host_Te, double *host_Tl, double *P0);
TTS_API int tts_set_ttm_state(tts_system *sys, int inst, const double *host_Te, const double *host_Tl);

/* Switch on the moving lattice (before tts_set_ttm_grid; general engine only).
 * From then on tts_step(n) advances n lattice steps and observables are
 * sampled every sample_every lattice steps, with [16] the ion kinetic
 * temperature, [17] the kinetic and [18] the pair-potential energy.
 * Errors: TTS_ERR_ARG, TTS_ERR_STATE (TTM grid already set),
 * TTS_ERR_UNSUPPORTED (cluster or a fast engine). */
TTS_API int tts_set_lattice(tts_system *sys, const tts_lattice_desc *lat);
/* Positions (angstrom, wrapped into the box) and velocities (m/s) of one
 * instance, canonical order. */
TTS_API int tts_get_positions(tts_system *sys, int inst, double *host_xyz);
TTS_API int tts_get_velocities(tts_system *sys, int inst, double *host_xyz);

/* The step counter (the Philox step word and the time t = step * dt). */
TTS_API int tts_get_step(tts_system *sys, int64_t *step);
TTS_API int tts_set_step(tts_system *sys, int64_t step);

/* Checkpoint: every piece of dynamic state (spins, TTM grids, step counter,
 * observable rings) in an opaque byte string.  With buf == NULL, *nbytes
 * receives the size needed.  Restoring into a system created from the same
 * description and continuing reproduces an uninterrupted run bit for bit. */
TTS_API int tts_get_state(tts_system *sys, void *buf, size_t *nbytes);
TTS_API int tts_set_state(tts_system *sys, const void *buf, size_t nbytes);

TTS_API int tts_info(tts_system *sys, tts_info_t *info);

/* Kernel timing.  While enabled, tts_step records each call's steps, with
 * CUDA events around every step's dominant kernels (the colour passes, or
 * the fused step kernel of a fast engine), into a graph of their own (every
 * kernel a node, none of the cached step graphs) and replays it on the
 * system's stream, waiting for it before it returns; the resident engine
 * brackets its multi-step launch instead.  No work is skipped and the results
 * are those of the unprofiled path. */
TTS_API int tts_profile_enable(tts_system *sys, int enable);
/* Total duration in ms of the bracketed kernels since profiling was enabled,
 * the number of steps bracketed, and the spin-steps those steps completed
 * (atoms x steps).  Synchronises the stream. */
TTS_API int tts_profile_read(tts_system *sys, double *ms, int64_t *steps, int64_t *spin_steps);

/* Largest grid (cells) that tts_ttm_advance_noalloc() accepts. */
#define TTS_NOALLOC_MAX_CELLS 65536

/* Advance one two-temperature grid held in the caller's device buffers by
 * one time step dt (from t = step * dt), without allocating any memory.
 * The paper has no counterpart: this is a convenience for callers that cannot
 * allocate device memory, such as code whose device memory is entirely owned
 * by another allocator (a framework's caching pool) or latency-critical code
 * that must not call cudaMalloc / cudaFree, which can synchronise the device.
 * The update is that of tts_step's TTM grid (explicit FTCS of the electron
 * energy, periodic Laplacian, e-ph exchange, Gaussian source with the spatial
 * profile of `t`), except that no calibration is done: the source power is
 * t->P0 for any source kind other than TTS_SOURCE_NONE, with pulse width
 * t->fwhm.  box_ang: grid box edges in angstrom.  dev_Te, dev_Tl: device
 * arrays of t->cells[0]*t->cells[1]*t->cells[2] doubles (x fastest), updated
 * in place.  dev_deposited: NULL or one device double that receives the
 * source energy (J) deposited by this call.  stream: cudaStream_t or NULL.
 * Scratch lives in a fixed device array of TTS_NOALLOC_MAX_CELLS doubles
 * (512 KiB) that every GPU loading this library holds until the process
 * exits; larger grids are rejected with TTS_ERR_ARG.  The first call on each
 * device looks the array's device address up (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  All calls on one GPU share that
 * GPU's array and find in it whatever the previous call left (nothing has to
 * start at zero): calls that overlap on the same GPU, for example on two
 * streams, race on it and give wrong results.  Asynchronous: returns once queued.
 * Errors: TTS_ERR_ARG, TTS_ERR_CUDA, TTS_ERR_UNSUPPORTED (device index > 63). */
TTS_API int tts_ttm_advance_noalloc(const tts_ttm_desc *t, const double box_ang[3], double dt, int64_t step,
                                    double *dev_Te, double *dev_Tl, double *dev_deposited, void *stream);

/* Autotuner: time every launch configuration the system's engine offers
 * (block shapes of the colour-pass kernels, the instance chains of the FP32
 * checker's separate passes, the fused sweep at each fusion depth; threads
 * per CTA of the resident kernel) over probe_steps steps each, starting every probe from the same
 * saved state and restoring it afterwards, and keep the fastest.  Choices are
 * cached per engine, precision and shape for the life of the process.
 * *chosen (may be NULL) receives the index of the configuration kept and
 * *n_configs the number offered.  Results of later steps do not depend on the
 * choice.  Errors: TTS_ERR_ARG, TTS_ERR_STATE (profiling on), TTS_ERR_CUDA. */
TTS_API int tts_autotune(tts_system *sys, int probe_steps, int *chosen, int *n_configs);

/* Select launch configuration `index` (0 .. n_configs - 1, the order the
 * autotuner tries them; 0 is the engine's default) without timing anything.
 * index < 0 only reports: *n_configs (may be NULL) receives the number offered
 * and *current (may be NULL) the index in use.  Results do not depend on the
 * choice.  Errors: TTS_ERR_ARG (index out of range). */
TTS_API int tts_set_config(tts_system *sys, int index, int *current, int *n_configs);

/* Message of the calling thread's last failed call (never NULL). */
TTS_API const char *tts_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTS_H */
