// tts_kernels.h -- launchers of the device kernels (implemented in tts_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "tts_internal.h"

namespace tts {

// Parameters passed by value to every step kernel.
struct StepParams {
    SpeciesParams sp[TTS_MAX_SPECIES];
    double axis[3];
    double B[3];
    double dt;
    uint32_t key0, key1;
    int nspecies;
    int64_t n_total;         // slots
    int zmax;                // neighbour-table width (general engine)
    int n_instances;
    int instance_base;       // global id of instance 0 (Philox counter word 3)
    int sample_every;
    int obs_capacity;
    int ncells_total;        // TTM cells over all instances (host-side launch size)
    int obs_blocks;          // observable partial blocks (host-side launch size)
    int ttm_one_substep;     // every TTM grid advances in one sub-step per step
    int sigma_per_step;      // the noise table is rebuilt by its own kernel every step
    int lattice_on;          // observables of a moving lattice (sampled per lattice step)
    int merged;              // merged (leapfrog) sweep (engines read it from here)
    int obs_skip;            // host-side: record this step without its observable kernels
                             // (a step the host knows does not sample)
    int sigma_alternate;     // the TTM of this step runs beside its colour passes: it writes
                             // the next step's noise table into the other of sigma / sigma_alt
                             // (by the parity of that step) and leaves the step counter alone
    int sigma_parity;        // with sigma_alternate: the parity of this step (fixed when the
                             // step is recorded; its graph is replayed only at that parity)
    int64_t *lstep;          // lattice step counter (moving lattice)
    double *lat_partial;     // per observable block: kinetic and pair energy (moving lattice)
};

// Device buffers of a system (general engine layout, real_t = float or double).
struct DevBuffers {
    void *sx = nullptr, *sy = nullptr, *sz = nullptr;   // spins, slot order
    int *atom = nullptr;          // canonical atom id of each slot
    uint8_t *species = nullptr;   // species of each slot
    int *cell = nullptr;          // global TTM cell of each slot
    int *nbr = nullptr;           // zmax * n_total neighbour slots (column-major)
    void *nbr_w = nullptr;        // zmax * n_total J_ij / mu_i (tesla), real_t
    void *sigma = nullptr;        // ncells * 2 species * 2 (h = dt/2, dt), real_t
    void *sigma_alt = nullptr;    // a second table of the same shape, right after sigma in its
                                  // allocation: with sigma_alternate the table of step n is
                                  // sigma (n even) or sigma_alt (n odd)
    double *Te = nullptr, *Tl = nullptr;   // per global cell
    double *src_shape = nullptr;  // per global cell
    double *ttm_scratch = nullptr;// 2 * ncells
    double *src_energy = nullptr; // per instance, J
    DevInstance *inst = nullptr;  // per instance
    PassRange *ranges = nullptr;  // concatenated over passes
    int64_t *step = nullptr;      // device step counter
    int *open = nullptr;          // merged sweep: colour 0 is half a step ahead
    int64_t *target = nullptr;    // merged sweep: step count at the end of the current call
    unsigned int *health = nullptr;
    double *obs_partial = nullptr;// per observable block, kObsFields doubles
    int *obs_block_inst = nullptr;// instance of each observable block
    int64_t *obs_block_begin = nullptr; // first slot of each observable block
    double *obs_ring = nullptr;   // n_instances * capacity * TTS_NOBS
    int64_t *obs_count = nullptr; // samples taken per instance
    double *obs_now = nullptr;    // n_instances * TTS_NOBS
    int *cell_inst = nullptr;     // instance of each TTM cell
};

// Merged-sweep control of a colour-0 pass (the splitting of paper Sec. II.A in
// leapfrog form).  mode 0: h fixed by the launch; 1: the leading pass, h = dt
// (a bridge) when the previous step left colour 0 open, else dt/2; 2: the
// trailing half-pass, run only when the step closes -- a sampling step or the
// last step of the call -- and recording for the next step whether it did.
struct SweepCtl {
    int mode = 0;
    int *open = nullptr;
    const int64_t *target = nullptr;
    int sample_every = 0;
};

#ifdef __CUDACC__
// Apply the control: returns false when the (trailing) pass is skipped;
// sets hsel for a leading pass.  Every thread of the launch gets the same
// answer; block 0's thread 0 records the open state.
__device__ __forceinline__ bool sweep_gate(const SweepCtl &w, const int64_t *step, int &hsel)
{
    if (w.mode == 1) {
        hsel = *w.open ? 1 : 0;
        return true;
    }
    if (w.mode == 2) {
        const int64_t n = *step;
        const bool close = (w.sample_every > 0 && (n + 1) % w.sample_every == 0) || n + 1 == *w.target;
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
            *w.open = close ? 0 : 1;
        return close;
    }
    return true;
}
#endif

constexpr int kObsFields = 24;       // per species: 12 partial sums
constexpr int kObsBlock = 128;       // threads of an observable block
constexpr int kObsSpan = 1024;       // slots of an observable block (8 a thread)

#ifdef __CUDACC__
// Sum v over the block's kObsBlock threads into out[k] for k < NF: shuffles within each
// warp, then warp 0's lanes add the warps' sums in warp order (a fixed order,
// so the result does not depend on timing).
template <int NF>
__device__ __forceinline__ void block_sum_store(const double (&v)[NF], double *out)
{
    __shared__ double wsum[kObsBlock / 32][NF];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) wsum[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kObsBlock / 32; ++w) t += wsum[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}
#endif

enum HealthBits : unsigned int {
    kHealthNonFinite = 1u,
    kHealthTimeout = 2u,
    kHealthSkin = 4u,        // an atom left its neighbour-list skin
    kHealthColour = 8u,      // two exchange-coupled atoms share a colour
    kHealthOverflow = 16u,   // more exchange neighbours than the table holds
};

cudaError_t launch_sigma(const StepParams &p, const DevBuffers &b, int ncells_total, int precision,
                         cudaStream_t st);
cudaError_t launch_pass_general(const StepParams &p, const DevBuffers &b, int precision, int pass,
                                int64_t range_offset, int nranges, int64_t nwork, cudaStream_t st, int block = 256,
                                SweepCtl sw = SweepCtl());
// target = step + n (merged sweep: the call's last step closes)
cudaError_t launch_set_target(const DevBuffers &b, int64_t n, cudaStream_t st);
// TTM advance of every instance; with one sub-step per step the grid-parallel
// path also refreshes the noise table for the next step and, with inc_step,
// advances the step counter.
cudaError_t launch_ttm(const StepParams &p, const DevBuffers &b, const TtmParams &tp, int n_instances,
                       cudaStream_t st, int precision, int inc_step);
cudaError_t launch_step_inc(const DevBuffers &b, cudaStream_t st);
// partials_done: the engine has written this step's observable partial sums.
cudaError_t step_tail(const StepParams &p, const DevBuffers &b, const TtmParams &tp, bool ttm_active, int n_inst,
                      int precision, int obs_blocks, cudaStream_t st, int *kernels, bool partials_done = false);
cudaError_t launch_obs(StepParams p, const DevBuffers &b, int precision, int nblocks, int mode, cudaStream_t st);
// General SoA (slot order) <-> xyz interleaved in canonical atom order of
// every instance (global index = slot_begin of the slot's instance + atom id).
cudaError_t launch_spins_to_atoms(const DevBuffers &b, int64_t n_total, int n_inst, int precision, void *out,
                                  cudaStream_t st);
cudaError_t launch_spins_from_atoms(const DevBuffers &b, int64_t n_total, int n_inst, int precision, const void *in,
                                    cudaStream_t st);
// The per-instance reduction of the partial sums (and, mode 0, the step
// increment) alone.
cudaError_t launch_obs_reduce(const StepParams &p, const DevBuffers &b, int mode, cudaStream_t st);

// Source-power calibration: P0 such that the largest T_e over the cells and
// the step times t_n of a TTM-only run (to t0 + 10 sigma_t) equals the target.
// Each launch evaluates ncand candidate powers per job, one CTA each; the host
// narrows the bracket (multi-section) until it is at double resolution.
struct CalibJob {
    int cells[3];
    int substeps;
    double dx[3];
    double sigma_t, t0;
    int64_t nsteps;            // step times to scan
    const double *shape;       // per cell source profile (device)
    double *work;              // ncand * 3 * ncells doubles of device scratch
};

cudaError_t launch_calibrate(const CalibJob *jobs_dev, const double *cand_dev, double *peaks_dev, int njobs,
                             int ncand, int ncells, double dt, const TtmParams &tp, cudaStream_t st);

}  // namespace tts
