// tts_schedule.h -- which captured step graph to replay for each stretch of
// steps while observables are sampled every `every` steps.
//
// Step n (the counter before the step) samples when (n + 1) % every == 0, the
// last step of each sampling interval.  A graph that records the observable
// kernels into every step pays for their launches at every step, although
// they return at once on all but one step in `every`; so the host keeps its
// own copy of the step counter and replays
//   Cycle    -- `every` steps starting at a multiple of `every`: the observable
//               kernels in the last step only,
//   PlainRun -- `run_len` steps without observable kernels,
//   Plain    -- one step without them,
//   Sample   -- one step with them,
// such that every sampling step runs in a graph that has them.  The kernels
// still test the device counter themselves, so a host copy that has drifted
// can misplace a sample but never the step count: every graph advances the
// counter by one per step.
//
// Plain host C++, no CUDA: the runtime and a host-side test both include it.
#pragma once
#include <cstdint>

namespace tts {

enum class StepGraph { Sample, Plain, PlainRun, Cycle };

// Emit the graph launches covering steps [step0, step0 + nsteps) in order.
// every >= 1; run_len >= 1 (steps in a PlainRun graph); cycle_len is `every`
// when a Cycle graph exists, else 0.  emit(kind, steps) is called per launch.
template <class Emit>
void schedule_steps(int64_t step0, int64_t nsteps, int64_t every, int64_t run_len, int64_t cycle_len, Emit &&emit)
{
    int64_t st = step0, left = nsteps;
    while (left > 0) {
        const int64_t phase = ((st % every) + every) % every;
        if (cycle_len > 0 && phase == 0 && left >= cycle_len) {
            emit(StepGraph::Cycle, cycle_len);
            st += cycle_len;
            left -= cycle_len;
            continue;
        }
        const int64_t plain = every - 1 - phase;   // steps before the next sampling step
        if (plain == 0) {
            emit(StepGraph::Sample, int64_t(1));
            ++st;
            --left;
            continue;
        }
        int64_t run = plain < left ? plain : left;
        for (; run >= run_len; run -= run_len, st += run_len, left -= run_len) emit(StepGraph::PlainRun, run_len);
        for (; run > 0; --run, ++st, --left) emit(StepGraph::Plain, int64_t(1));
    }
}

}  // namespace tts
