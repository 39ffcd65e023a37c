// tts_engines.cu -- fast engines.  None is available yet: every system runs
// on the general engine.
#include "tts_engines.h"

namespace tts {

struct EngineState {
    int unused;
};

int engine_select(const tts_system_desc &, const std::vector<HostInstance> &, int) { return -1; }
int engine_create(const tts_system_desc &, const std::vector<HostInstance> &, const std::vector<std::vector<int64_t>> &,
                  const std::vector<DevInstance> &, const StepParams &, const DevBuffers &, int, cudaStream_t,
                  EngineState **out)
{
    *out = nullptr;
    return TTS_ERR_UNSUPPORTED;
}
void engine_destroy(EngineState *e) { delete e; }
const char *engine_last_error() { return "no fast engine"; }
cudaError_t engine_record_step(EngineState *, const StepParams &, const DevBuffers &, const TtmParams &, bool,
                               cudaStream_t, int *, cudaEvent_t, cudaEvent_t)
{
    return cudaErrorNotSupported;
}
int engine_read_spins(EngineState *, int, void *, void *, void *, cudaStream_t) { return TTS_ERR_UNSUPPORTED; }
int engine_write_spins(EngineState *, int, const void *, const void *, const void *, cudaStream_t)
{
    return TTS_ERR_UNSUPPORTED;
}
int engine_set_cells(EngineState *, const std::vector<DevInstance> &, const std::vector<int> &, cudaStream_t)
{
    return TTS_ERR_UNSUPPORTED;
}
cudaError_t engine_sync_to_general(EngineState *, const DevBuffers &, cudaStream_t) { return cudaSuccess; }
cudaError_t engine_sync_from_general(EngineState *, const DevBuffers &, cudaStream_t) { return cudaSuccess; }

}  // namespace tts
