// tts_system.h -- the system object behind the C ABI (runtime and lattice
// module) and the error helpers they share.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tts_engines.h"
#include "tts_internal.h"
#include "tts_kernels.h"

struct tts_system;

namespace tts {

int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
int upload(void *dst, const void *src, size_t bytes, cudaStream_t st, const char *what);

template <typename T>
int dev_alloc(T **ptr, size_t count, const char *what)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TTS_ERR_OOM, std::string("cudaMalloc of ") + what + " failed: " + cudaGetErrorString(e));
    }
    *ptr = static_cast<T *>(q);
    return TTS_OK;
}

struct LatticeState;   // moving lattice (tts_lattice.cu)
void lattice_destroy(LatticeState *L);
// Issue one lattice step (ev0/ev1, when set, bracket its kernels).
cudaError_t lattice_record_step(tts_system *s, cudaStream_t st, int *kernels, cudaEvent_t ev0,
                                cudaEvent_t ev1);
int64_t lattice_units_per_step(const tts_system *s);
int lattice_refresh_now(tts_system *s);
int lattice_ensure_cell_acc(tts_system *s);
double lattice_step_length(const tts_system *s);
size_t lattice_state_bytes(const tts_system *s);
int lattice_state_io(tts_system *s, char *buf, bool save);
int lattice_refresh_tables(tts_system *s);

}  // namespace tts

#define TTS_CUDA(call, what)                                     \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return tts::cuda_fail(e_, what);  \
    } while (0)

struct tts_system {
    tts_system_desc desc{};
    int precision = 32;
    size_t rsize = 4;
    int engine = TTS_ENGINE_GENERAL;
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t capture = nullptr;    // private stream used only to capture graphs
    int64_t n_total = 0;
    int n_inst = 0;
    int zmax = 0;
    int max_colours = 1;
    int max_passes = 1;
    std::vector<tts::HostInstance> host;                 // built instances (canonical order)
    std::vector<std::vector<int64_t>> slot_of_atom; // per instance: atom -> slot (relative)
    std::vector<tts::DevInstance> dinst;
    std::vector<tts::PassRange> ranges;
    std::vector<int64_t> pass_offset;               // ranges of pass p: [off[p], off[p+1])
    std::vector<int64_t> pass_work;
    int ncells_total = 0;
    bool ttm_active = false;
    tts::TtmParams tp{};
    std::vector<double> P0;                         // per instance
    std::vector<double> inst_peak, inst_fwhm;       // per-instance pulse overrides (may be empty)
    int obs_blocks = 0;
    int obs_capacity = 1024;
    tts::DevBuffers b;
    tts::StepParams p{};
    // Step graphs, by the parity of the step they start at ([1] only when the
    // recorded steps depend on it: the noise tables alternated by parity)
    cudaGraphExec_t graph[2] = {};          // one step (with its observable kernels, if sampling)
    cudaGraphExec_t graph_multi[2] = {};    // graph_steps steps (without them, if sampling)
    cudaGraphExec_t graph_plain[2] = {};    // sampling only: one step without them
    cudaGraphExec_t graph_cycle[2] = {};    // sampling only: one sampling interval, them in its last step
    bool by_parity = false;                 // the [1] graphs exist
    int graph_steps = 16;
    int cycle_steps = 0;                    // steps of graph_cycle (0: none)
    int kernels_graph = 0, kernels_multi = 0, kernels_plain = 0, kernels_cycle = 0;   // per replay
    bool phased = false;                    // the graphs follow the sampling phase (above)
    int64_t host_step = 0;                  // host copy of the device step counter
    int64_t launches = 0;
    bool dirty = true;
    tts::EngineState *eng = nullptr;                     // fast-engine state, if any
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;           // begin/end pairs of profiled launches
    std::vector<int64_t> prof_pair_steps;           // steps covered by each pair
    double prof_ms = 0.0;
    int64_t prof_steps = 0;
    tts::LatticeState *lat = nullptr;               // moving lattice, if switched on
    int pass_block = 256;                           // general engine: threads per pass CTA
    std::vector<int> pass_blocks = {128, 256, 512}; // general engine: autotuner candidates
    void *io_buf = nullptr;                         // bulk spin I/O staging, 3 n_total reals
    bool merged = false;                            // merged (leapfrog) sweep in use
    bool merged_uniform = true;                     // every instance has the same colour count
};

