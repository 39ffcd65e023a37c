// tts_engines.h -- hooks of the fast engines (checkerboard and resident).
//
// The general engine keeps the canonical device state (slot-ordered spin
// arrays, TTM grids, observables).  A fast engine may keep spins in its own
// layout; it then provides the step recording and the spin transfers below,
// and copies its spins into the general arrays when observables or
// checkpoints need them.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "tts_internal.h"
#include "tts_kernels.h"

namespace tts {

struct EngineState;

// Returns the engine that will run the system (TTS_ENGINE_*), or -1 when the
// requested engine (or, for AUTO, every fast engine) cannot run it.
int engine_select(const tts_system_desc &d, const std::vector<HostInstance> &host, int requested);

int engine_create(const tts_system_desc &d, const std::vector<HostInstance> &host,
                  const std::vector<std::vector<int64_t>> &slot_of_atom, const std::vector<DevInstance> &dinst,
                  const StepParams &p, const DevBuffers &b, int engine, cudaStream_t st, EngineState **out);
void engine_destroy(EngineState *e);
const char *engine_last_error();

// Issue the kernels of one step on stream st (captured into a graph, or run
// directly while profiling).  ev_begin / ev_end, when not null, are recorded
// around the step's dominant kernels.
cudaError_t engine_record_step(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                               bool ttm_active, cudaStream_t st, int *kernels, cudaEvent_t ev_begin,
                               cudaEvent_t ev_end);
// The steps this engine records differ by the parity of their step (the TTM
// beside the colour passes, on noise tables alternated by parity): a recorded
// step is replayed only at the parity StepParams::sigma_parity names.
bool engine_step_parity(const EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                        bool ttm_active);
// Engines that advance many steps in one launch (resident): run nsteps steps.
bool engine_multi_step(const EngineState *e);
cudaError_t engine_run_steps(EngineState *e, const StepParams &p, const DevBuffers &b, const TtmParams &tp,
                             bool ttm_active, int64_t nsteps, cudaStream_t st, int *kernels, cudaEvent_t ev_begin,
                             cudaEvent_t ev_end);
// A TTM grid was attached (the cell map of every slot is in DevBuffers::cell).
int engine_set_cells(EngineState *e, const std::vector<DevInstance> &dinst, const std::vector<int> &cellmap,
                     cudaStream_t st);
// Launch configurations the engine offers to the autotuner.
int engine_num_configs(const EngineState *e);
void engine_set_config(EngineState *e, int index);
int engine_config(const EngineState *e);

cudaError_t engine_sync_to_general(EngineState *e, const DevBuffers &b, cudaStream_t st);
// Observable partial sums (the general kernel's per-block layout) straight
// from the engine's own spin layout; cudaErrorNotSupported when the engine
// has none.  mode 0: only on sampling steps; 1: now.
cudaError_t engine_obs_partials(EngineState *e, const StepParams &p, const DevBuffers &b, int mode, cudaStream_t st);
cudaError_t engine_sync_from_general(EngineState *e, const DevBuffers &b, cudaStream_t st);

}  // namespace tts
