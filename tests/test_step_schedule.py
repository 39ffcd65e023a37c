"""Host-side schedule of captured step graphs while observables are sampled
(csrc/tts_schedule.h), compiled with the host C++ compiler and checked here.

Rule (Sec. 2.4 sampling of the observables every k steps): step n, counted
before the step, samples when (n + 1) % k == 0.  The schedule must cover every
step exactly once, in order, and replay the observable kernels in exactly the
sampling steps, from any starting step.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2608_18541_b300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <initializer_list>
#include "tts_schedule.h"
using namespace tts;

// Expand the schedule into per-step flags (1 = observable kernels recorded in
// that step) and check them against the sampling rule.
static int check(int64_t step0, int64_t nsteps, int64_t every, int64_t run_len, int64_t cycle_len, int64_t *launches)
{
    int64_t st = step0, cycles = 0, n = 0;
    int bad = 0;
    schedule_steps(step0, nsteps, every, run_len, cycle_len, [&](StepGraph g, int64_t steps) {
        ++n;
        if (g == StepGraph::Cycle) {
            ++cycles;
            if (steps != cycle_len || st % every != 0) bad = 1;
        } else if (g == StepGraph::PlainRun) {
            if (steps != run_len) bad = 2;
        } else if (steps != 1) {
            bad = 3;
        }
        for (int64_t i = 0; i < steps; ++i, ++st) {
            const bool obs = g == StepGraph::Sample || (g == StepGraph::Cycle && i == steps - 1);
            const bool want = (st + 1) % every == 0;
            if (obs != want) bad = 4;
        }
    });
    if (st != step0 + nsteps) bad = 5;
    *launches = n;
    return bad;
}

int main()
{
    int64_t n = 0;
    const int64_t everies[] = {1, 2, 3, 5, 7, 16, 17, 100, 257, 1000};
    for (int64_t every : everies)
        for (int64_t run_len : {1, 4, 16})
            for (int cyc = 0; cyc < 2; ++cyc)
                for (int64_t step0 = 0; step0 < 2 * every + 3; step0 += (every > 40 ? 13 : 1))
                    for (int64_t nsteps : {1, 2, 3, 15, 16, 17, 99, 100, 101, 250, 1001}) {
                        const int64_t cycle_len = cyc ? every : 0;
                        const int b = check(step0, nsteps, every, run_len, cycle_len, &n);
                        if (b) {
                            std::printf("FAIL %d every=%lld run=%lld cycle=%lld step0=%lld n=%lld\n", b,
                                        (long long)every, (long long)run_len, (long long)cycle_len,
                                        (long long)step0, (long long)nsteps);
                            return 1;
                        }
                    }
    // benchmark pattern: 100-step calls aligned to a 100-step interval are one replay each
    for (int64_t call = 0; call < 5; ++call) {
        if (check(100 * call, 100, 100, 16, 100, &n) || n != 1) {
            std::printf("FAIL aligned call %lld launches %lld\n", (long long)call, (long long)n);
            return 1;
        }
    }
    // no cycle graph: 99 plain steps in runs of 16 and singles, then the sampling step
    if (check(0, 100, 100, 16, 0, &n) || n != 6 + 3 + 1) {
        std::printf("FAIL plain runs %lld\n", (long long)n);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp(prefix="tts_sched_")
    src = os.path.join(d, "drv.cpp")
    exe = os.path.join(d, "drv")
    with open(src, "w") as f:
        f.write(DRIVER)
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", CSRC, src, "-o", exe])
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def test_schedule_covers_every_step_and_samples_exactly(driver):
    out = subprocess.run([driver], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "OK"
