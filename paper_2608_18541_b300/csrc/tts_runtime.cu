// tts_runtime.cu -- the C ABI of include/tts.h: system construction, device
// memory, the captured per-step CUDA graph, TTM set-up and calibration,
// observables, checkpoints.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "tts_bulk.cuh"
#include "tts_engines.h"
#include "tts_internal.h"
#include "tts_kernels.h"
#include "tts_schedule.h"
#include "tts_system.h"

using namespace tts;

namespace {
thread_local std::string g_error = "no error";
}  // namespace

void tts::set_last_error(const std::string &msg) { g_error = msg; }

int tts::fail(int code, const std::string &msg)
{
    g_error = msg;
    return code;
}

int tts::cuda_fail(cudaError_t e, const char *what)
{
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TTS_ERR_OOM : TTS_ERR_CUDA;
}

int tts::upload(void *dst, const void *src, size_t bytes, cudaStream_t st, const char *what)
{
    if (bytes == 0) return TTS_OK;
    TTS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), what);
    TTS_CUDA(cudaStreamSynchronize(st), what);
    return TTS_OK;
}



namespace {

void free_buffers(tts_system *s)
{
    DevBuffers &b = s->b;
    void *ptrs[] = {b.sx, b.sy, b.sz, b.atom, b.species, b.cell, b.nbr, b.nbr_w, b.sigma, b.Te, b.Tl,
                    b.src_shape, b.ttm_scratch, b.src_energy, b.inst, b.ranges, b.step, b.health,
                    b.obs_partial, b.obs_block_inst, b.obs_block_begin, b.obs_ring, b.obs_count, b.obs_now,
                    b.cell_inst, b.open, b.target};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    s->b = DevBuffers{};
}


int validate(const tts_system_desc &d)
{
    if (d.nspecies < 1 || d.nspecies > TTS_MAX_SPECIES) return fail(TTS_ERR_ARG, "nspecies must be 1 or 2");
    if (d.precision != 32 && d.precision != 64) return fail(TTS_ERR_ARG, "precision must be 32 or 64");
    if (!(d.dt > 0.0)) return fail(TTS_ERR_ARG, "dt must be positive");
    if (d.n_instances < 1) return fail(TTS_ERR_ARG, "n_instances must be >= 1");
    if (d.lattice < 0 || d.lattice > 3) return fail(TTS_ERR_ARG, "unknown lattice");
    if (d.lattice != TTS_LATTICE_CLUSTER && !(d.a > 0.0)) return fail(TTS_ERR_ARG, "lattice constant must be positive");
    if (d.lattice == TTS_LATTICE_CLUSTER && d.n_instances != 1)
        return fail(TTS_ERR_ARG, "explicit clusters take one instance");
    for (int t = 0; t < d.nspecies; ++t) {
        if (!(d.mu_muB[t] > 0.0)) return fail(TTS_ERR_ARG, "moments must be positive");
        if (!(d.alpha[t] >= 0.0)) return fail(TTS_ERR_ARG, "damping must be >= 0");
        const double *v = d.init_dir[t];
        if (!(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] > 0.0)) return fail(TTS_ERR_ARG, "zero initial direction");
    }
    for (int a = 0; a < d.nspecies; ++a)
        for (int c = 0; c < d.nspecies; ++c) {
            const tts_exchange &x = d.exch[a][c], &y = d.exch[c][a];
            if (x.kind < 0 || x.kind > 2) return fail(TTS_ERR_ARG, "unknown exchange kind");
            if (x.kind != y.kind || x.J1 != y.J1 || x.J2 != y.J2 || x.J3 != y.J3 || x.rc != y.rc)
                return fail(TTS_ERR_ARG, "exchange table must be symmetric");
            if (x.kind == TTS_EXCH_BETHE_SLATER && !(x.J3 > 0.0)) return fail(TTS_ERR_ARG, "J3 must be positive");
        }
    if (!(d.T_bath >= 0.0)) return fail(TTS_ERR_ARG, "T_bath must be >= 0");
    if (d.inst_T_bath)
        for (int i = 0; i < d.n_instances; ++i)
            if (!(d.inst_T_bath[i] >= 0.0)) return fail(TTS_ERR_ARG, "instance bath temperatures must be >= 0");
    if (d.engine < 0 || d.engine > 3) return fail(TTS_ERR_ARG, "unknown engine");
    if (d.sample_every < 0) return fail(TTS_ERR_ARG, "sample_every must be >= 0");
    if (d.instance_base < 0) return fail(TTS_ERR_ARG, "instance_base must be >= 0");
    if (d.sweep != TTS_SWEEP_SYMMETRIC && d.sweep != TTS_SWEEP_MERGED) return fail(TTS_ERR_ARG, "unknown sweep");
    return TTS_OK;
}

// ---------------------------------------------------------------------------
// TTM set-up on the host: cell of each atom, source shape, sub-steps and the
// calibration of P0 (bisection on a TTM-only run).
// ---------------------------------------------------------------------------
struct HostTtm {
    int cells[3];
    double dx[3], vol;
    int substeps;
    double sigma_t, t0;
    std::vector<double> shape;
};

int make_host_ttm(double step_dt, const HostInstance &hi, const tts_ttm_desc &t, double fwhm, HostTtm *o)
{
    int resolved = 0;
    double dxmin = 0.0;
    o->vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        o->cells[k] = t.cells[k];
        o->dx[k] = hi.box[k] * kAngstrom / t.cells[k];
        o->vol *= o->dx[k];
        if (t.cells[k] > 1) {
            dxmin = resolved ? std::min(dxmin, o->dx[k]) : o->dx[k];
            ++resolved;
        }
    }
    o->substeps = 1;
    if (resolved > 0 && t.kappa_e > 0.0) {
        const double limit = 0.4 * t.gamma_e * t.T0 * dxmin * dxmin / (t.kappa_e * resolved);
        const double m = std::ceil(step_dt / limit);
        o->substeps = m < 1.0 ? 1 : static_cast<int>(m);
    }
    o->sigma_t = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    o->t0 = t.t0 >= 0.0 ? t.t0 : 3.0 * o->sigma_t;
    const int nc = t.cells[0] * t.cells[1] * t.cells[2];
    o->shape.assign(nc, 1.0);
    for (int cz = 0; cz < t.cells[2]; ++cz)
        for (int cy = 0; cy < t.cells[1]; ++cy)
            for (int cx = 0; cx < t.cells[0]; ++cx) {
                const int c = (cz * t.cells[1] + cy) * t.cells[0] + cx;
                const double x = (cx + 0.5) * hi.box[0] / t.cells[0];
                const double y = (cy + 0.5) * hi.box[1] / t.cells[1];
                const double z = (cz + 0.5) * hi.box[2] / t.cells[2];
                if (t.spatial == TTS_SPATIAL_XY_GAUSS) {
                    const double rx = x - 0.5 * hi.box[0], ry = y - 0.5 * hi.box[1];
                    o->shape[c] = std::exp(-(rx * rx + ry * ry) / (2.0 * t.sigma_xy * t.sigma_xy));
                } else if (t.spatial == TTS_SPATIAL_Z_EXP) {
                    o->shape[c] = std::exp(-z / t.depth_z);
                }
            }
    return TTS_OK;
}

// ---------------------------------------------------------------------------
// General-engine layout and upload
// ---------------------------------------------------------------------------
template <typename R>
int upload_general(tts_system *s)
{
    const int64_t N = s->n_total;
    std::vector<int> atom(N), cell(N), nbr(size_t(s->zmax) * N);
    std::vector<uint8_t> spc(N);
    std::vector<R> w(size_t(s->zmax) * N), sx(N), sy(N), sz(N);
    for (int i = 0; i < s->n_inst; ++i) {
        const HostInstance &hi = s->host[i];
        const DevInstance &di = s->dinst[i];
        for (int64_t a = 0; a < hi.n; ++a) {
            const int64_t slot = di.slot_begin + s->slot_of_atom[i][a];
            atom[slot] = static_cast<int>(a);
            spc[slot] = hi.species[a];
            cell[slot] = di.cell_begin;  // uniform bath: one cell per instance until a TTM grid is set
            const double inv_mu = 1.0 / (s->desc.mu_muB[hi.species[a]] * kBohrMagneton);
            const int64_t b0 = hi.nbr_begin[a], b1 = hi.nbr_begin[a + 1];
            for (int k = 0; k < s->zmax; ++k) {
                const size_t e = size_t(k) * N + slot;
                if (b0 + k < b1) {
                    nbr[e] = static_cast<int>(di.slot_begin + s->slot_of_atom[i][hi.nbr[b0 + k]]);
                    w[e] = static_cast<R>(hi.nbr_J[b0 + k] * inv_mu);
                } else {
                    nbr[e] = static_cast<int>(slot);
                    w[e] = R(0);
                }
            }
            const double *v = s->desc.init_dir[hi.species[a]];
            const double m = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            sx[slot] = static_cast<R>(v[0] / m);
            sy[slot] = static_cast<R>(v[1] / m);
            sz[slot] = static_cast<R>(v[2] / m);
        }
    }
    DevBuffers &b = s->b;
    int rc;
    if ((rc = upload(b.atom, atom.data(), N * sizeof(int), s->stream, "upload atom ids"))) return rc;
    if ((rc = upload(b.species, spc.data(), N, s->stream, "upload species"))) return rc;
    if ((rc = upload(b.cell, cell.data(), N * sizeof(int), s->stream, "upload cells"))) return rc;
    if ((rc = upload(b.nbr, nbr.data(), nbr.size() * sizeof(int), s->stream, "upload neighbours"))) return rc;
    if ((rc = upload(b.nbr_w, w.data(), w.size() * sizeof(R), s->stream, "upload couplings"))) return rc;
    if ((rc = upload(b.sx, sx.data(), N * sizeof(R), s->stream, "upload spins"))) return rc;
    if ((rc = upload(b.sy, sy.data(), N * sizeof(R), s->stream, "upload spins"))) return rc;
    if ((rc = upload(b.sz, sz.data(), N * sizeof(R), s->stream, "upload spins"))) return rc;
    return TTS_OK;
}

int alloc_cells(tts_system *s, int ncells_total)
{
    DevBuffers &b = s->b;
    for (void *q : {(void *)b.Te, (void *)b.Tl, (void *)b.src_shape, (void *)b.ttm_scratch, b.sigma,
                    (void *)b.cell_inst})
        if (q) cudaFree(q);
    b.Te = b.Tl = b.src_shape = b.ttm_scratch = nullptr;
    b.sigma = b.sigma_alt = nullptr;
    b.cell_inst = nullptr;
    int rc;
    if ((rc = dev_alloc(&b.Te, ncells_total, "T_e"))) return rc;
    if ((rc = dev_alloc(&b.Tl, ncells_total, "T_l"))) return rc;
    if ((rc = dev_alloc(&b.src_shape, ncells_total, "source shape"))) return rc;
    if ((rc = dev_alloc(&b.ttm_scratch, 2 * size_t(ncells_total), "TTM scratch"))) return rc;
    if ((rc = dev_alloc(&b.cell_inst, ncells_total, "cell instances"))) return rc;
    // the two noise tables (see DevBuffers::sigma_alt) in one allocation
    char *sig = nullptr;
    const size_t table = size_t(ncells_total) * TTS_MAX_SPECIES * 2 * s->rsize;
    if ((rc = dev_alloc(&sig, 2 * table, "sigma tables"))) return rc;
    b.sigma = sig;
    b.sigma_alt = sig + table;
    s->ncells_total = ncells_total;
    s->p.ncells_total = ncells_total;
    return TTS_OK;
}

// Issue the kernels of one step on stream c.  ev0 / ev1 (may be null) are
// recorded around the dominant kernels (the colour passes).
// Merged-sweep control of pass `pass` of `npass`: the first pass leads, the
// last trails; every other pass (and every pass of a symmetric sweep) is fixed.
SweepCtl sweep_ctl(const tts_system *s, int pass, int npass)
{
    SweepCtl w;
    if (!s->merged) return w;
    w.mode = pass == 0 ? 1 : (pass == npass - 1 ? 2 : 0);
    w.open = s->b.open;
    w.target = s->b.target;
    w.sample_every = s->p.sample_every;
    return w;
}

cudaError_t record_step(tts_system *s, cudaStream_t c, int *kernels, cudaEvent_t ev0, cudaEvent_t ev1, bool obs,
                        int64_t step)
{
    *kernels = 0;
    if (s->lat) return lattice_record_step(s, c, kernels, ev0, ev1);
    StepParams p = s->p;
    p.obs_skip = obs ? 0 : 1;
    p.sigma_parity = static_cast<int>(step & 1);
    if (s->eng) {
        p.merged = s->merged ? 1 : 0;
        return engine_record_step(s->eng, p, s->b, s->tp, s->ttm_active, c, kernels, ev0, ev1);
    }
    // general engine
    cudaError_t e = cudaSuccess;
    if (s->p.sigma_per_step) {
        e = launch_sigma(s->p, s->b, s->ncells_total, s->precision, c);
        ++*kernels;
    }
    if (e == cudaSuccess && ev0) e = cudaEventRecordWithFlags(ev0, c, cudaEventRecordExternal);
    for (int pass = 0; pass < s->max_passes && e == cudaSuccess; ++pass) {
        const int64_t off = s->pass_offset[pass];
        const int nr = static_cast<int>(s->pass_offset[pass + 1] - off);
        e = launch_pass_general(s->p, s->b, s->precision, pass, off, nr, s->pass_work[pass], c, s->pass_block,
                                sweep_ctl(s, pass, s->max_passes));
        ++*kernels;
    }
    if (e == cudaSuccess && ev1) e = cudaEventRecordWithFlags(ev1, c, cudaEventRecordExternal);
    e = (e == cudaSuccess) ? step_tail(p, s->b, s->tp, s->ttm_active, s->n_inst, s->precision, s->obs_blocks, c, kernels)
                           : e;
    return e;
}

void destroy_graphs(tts_system *s)
{
    for (cudaGraphExec_t *set : {s->graph, s->graph_multi, s->graph_plain, s->graph_cycle})
        for (int v = 0; v < 2; ++v)
            if (set[v]) {
                cudaGraphExecDestroy(set[v]);
                set[v] = nullptr;
            }
    s->by_parity = false;
}

// Capture nsteps steps into one graph, to be replayed from steps of the
// parity of step0.  obs: 0 = every step without its observable kernels, 1 =
// every step with them, 2 = only the last step with them.  *kernels_out =
// kernels per replay.
int capture_steps(tts_system *s, int nsteps, int obs, int64_t step0, cudaGraphExec_t *out, int *kernels_out)
{
    cudaStream_t c = s->capture;
    TTS_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "begin capture");
    int total = 0;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nsteps && e == cudaSuccess; ++i) {
        int kernels = 0;
        e = record_step(s, c, &kernels, nullptr, nullptr, obs == 1 || (obs == 2 && i == nsteps - 1), step0 + i);
        total += kernels;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "record step");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate step graph");
    *kernels_out = total;
    return TTS_OK;
}

// Longest sampling interval captured as one graph (about five kernels a step).
constexpr int kMaxCycleSteps = 256;

int build_graph(tts_system *s)
{
    destroy_graphs(s);
    // a moving lattice has ~100 kernels per step: fewer steps per graph
    s->graph_steps = s->lat ? 4 : 16;
    // While sampling, graphs follow the sampling phase (tts_schedule.h); a
    // moving lattice samples on its lattice clock and keeps the observable
    // kernels in every step.
    s->phased = !s->lat && s->p.sample_every > 0;
    s->cycle_steps = 0;
    StepParams q = s->p;
    q.merged = s->merged ? 1 : 0;
    s->by_parity = !s->lat && s->eng && engine_step_parity(s->eng, q, s->b, s->tp, s->ttm_active);
    const bool cycle = s->phased && s->p.sample_every >= 2 && s->p.sample_every <= kMaxCycleSteps;
    int rc = TTS_OK;
    for (int v = 0; v < (s->by_parity ? 2 : 1) && !rc; ++v) {
        rc = capture_steps(s, 1, 1, v, &s->graph[v], &s->kernels_graph);
        if (!rc) rc = capture_steps(s, s->graph_steps, s->phased ? 0 : 1, v, &s->graph_multi[v], &s->kernels_multi);
        if (!rc && s->phased) rc = capture_steps(s, 1, 0, v, &s->graph_plain[v], &s->kernels_plain);
        if (!rc && cycle) rc = capture_steps(s, s->p.sample_every, 2, v, &s->graph_cycle[v], &s->kernels_cycle);
    }
    if (cycle && !rc) s->cycle_steps = s->p.sample_every;
    if (rc) return rc;
    s->dirty = false;
    return TTS_OK;
}

void drop_profile_events(tts_system *s)
{
    for (cudaEvent_t ev : s->prof_events) cudaEventDestroy(ev);
    s->prof_events.clear();
    s->prof_pair_steps.clear();
}

}  // namespace

// End of a step for the general and checker engines: TTM, then either the
// observable kernels (which advance the step counter) or a bare increment,
// folded into the TTM update when that runs on the grid-parallel path.
cudaError_t tts::step_tail(const StepParams &p, const DevBuffers &b, const TtmParams &tp, bool ttm_active, int n_inst,
                           int precision, int obs_blocks, cudaStream_t st, int *kernels, bool partials_done)
{
    const bool sampling = p.sample_every > 0 && !p.obs_skip;
    const bool fold = ttm_active && p.ttm_one_substep && !sampling;
    cudaError_t e = cudaSuccess;
    if (ttm_active) {
        e = launch_ttm(p, b, tp, n_inst, st, precision, fold ? 1 : 0);
        *kernels += p.ttm_one_substep ? 2 : 1;
    }
    if (e != cudaSuccess) return e;
    if (sampling && partials_done) {
        e = launch_obs_reduce(p, b, 0, st);
        *kernels += 2;
    } else if (sampling) {
        e = launch_obs(p, b, precision, obs_blocks, 0, st);
        *kernels += 3;
    } else if (!fold) {
        e = launch_step_inc(b, st);
        *kernels += 1;
    }
    return e;
}

namespace {

// Noise table from the current T_e (after creation and every change of state
// that the per-step kernels do not see).
int refresh_sigma(tts_system *s)
{
    if (!s->b.sigma) return TTS_OK;
    cudaError_t e = launch_sigma(s->p, s->b, s->ncells_total, s->precision, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    ++s->launches;
    return e == cudaSuccess ? TTS_OK : cuda_fail(e, "noise table");
}

int check_inst(tts_system *s, int inst)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    if (inst < 0 || inst >= s->n_inst) return fail(TTS_ERR_ARG, "instance index out of range");
    return TTS_OK;
}

template <typename R>
int read_instance_spins(tts_system *s, int inst, double *out)
{
    const DevInstance &di = s->dinst[inst];
    std::vector<R> x(di.n), y(di.n), z(di.n);
    {
        if (s->eng) {
            cudaError_t e = engine_sync_to_general(s->eng, s->b, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "engine gather");
        }
        const size_t off = di.slot_begin * sizeof(R);
        TTS_CUDA(cudaMemcpyAsync(x.data(), static_cast<char *>(s->b.sx) + off, di.n * sizeof(R), cudaMemcpyDeviceToHost, s->stream), "read spins");
        TTS_CUDA(cudaMemcpyAsync(y.data(), static_cast<char *>(s->b.sy) + off, di.n * sizeof(R), cudaMemcpyDeviceToHost, s->stream), "read spins");
        TTS_CUDA(cudaMemcpyAsync(z.data(), static_cast<char *>(s->b.sz) + off, di.n * sizeof(R), cudaMemcpyDeviceToHost, s->stream), "read spins");
        TTS_CUDA(cudaStreamSynchronize(s->stream), "read spins");
    }
    const std::vector<int64_t> &so = s->slot_of_atom[inst];
    for (int64_t a = 0; a < di.n; ++a) {
        out[3 * a] = x[so[a]];
        out[3 * a + 1] = y[so[a]];
        out[3 * a + 2] = z[so[a]];
    }
    return TTS_OK;
}

template <typename R>
int write_instance_spins(tts_system *s, int inst, const double *in)
{
    const DevInstance &di = s->dinst[inst];
    std::vector<R> x(di.n), y(di.n), z(di.n);
    const std::vector<int64_t> &so = s->slot_of_atom[inst];
    for (int64_t a = 0; a < di.n; ++a) {
        const double vx = in[3 * a], vy = in[3 * a + 1], vz = in[3 * a + 2];
        const double m = std::sqrt(vx * vx + vy * vy + vz * vz);
        if (!(m > 0.0) || !std::isfinite(m)) return fail(TTS_ERR_ARG, "spin vectors must be finite and non-zero");
        x[so[a]] = static_cast<R>(vx / m);
        y[so[a]] = static_cast<R>(vy / m);
        z[so[a]] = static_cast<R>(vz / m);
    }
    if (s->eng) {
        // bring the general arrays up to date first: only this instance is overwritten below
        cudaError_t e = engine_sync_to_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine gather");
    }
    const size_t off = di.slot_begin * sizeof(R);
    TTS_CUDA(cudaMemcpyAsync(static_cast<char *>(s->b.sx) + off, x.data(), di.n * sizeof(R), cudaMemcpyHostToDevice, s->stream), "write spins");
    TTS_CUDA(cudaMemcpyAsync(static_cast<char *>(s->b.sy) + off, y.data(), di.n * sizeof(R), cudaMemcpyHostToDevice, s->stream), "write spins");
    TTS_CUDA(cudaMemcpyAsync(static_cast<char *>(s->b.sz) + off, z.data(), di.n * sizeof(R), cudaMemcpyHostToDevice, s->stream), "write spins");
    if (s->eng) {
        cudaError_t e = engine_sync_from_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine scatter");
    }
    TTS_CUDA(cudaStreamSynchronize(s->stream), "write spins");
    return TTS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *tts_last_error(void) { return g_error.c_str(); }

int tts_destroy(tts_system *s)
{
    if (!s) return TTS_OK;
    cudaStreamSynchronize(s->stream);
    destroy_graphs(s);
    drop_profile_events(s);
    if (s->eng) engine_destroy(s->eng);
    if (s->lat) lattice_destroy(s->lat);
    if (s->io_buf) cudaFree(s->io_buf);
    free_buffers(s);
    if (s->capture) cudaStreamDestroy(s->capture);
    delete s;
    return TTS_OK;
}

int tts_create_system(const tts_system_desc *desc, void *stream, tts_system **out)
{
    if (!out) return fail(TTS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(TTS_ERR_ARG, "desc is NULL");
    int rc = validate(*desc);
    if (rc) return rc;
    tts_system *raw = new (std::nothrow) tts_system;
    if (!raw) return fail(TTS_ERR_OOM, "host allocation failed");
    // on any early return the partly built system is released with tts_destroy
    struct Guard {
        tts_system *p;
        ~Guard() { if (p) tts_destroy(p); }
        tts_system *operator->() const { return p; }
        tts_system *get() const { return p; }
        tts_system *release() { tts_system *q = p; p = nullptr; return q; }
    } s{raw};
    s->desc = *desc;
    s->precision = desc->precision;
    s->rsize = desc->precision == 64 ? 8 : 4;
    s->stream = static_cast<cudaStream_t>(stream);
    s->n_inst = desc->n_instances;
    s->obs_capacity = desc->obs_capacity > 0 ? desc->obs_capacity : 1024;
    // host build (all argument errors are found here, before any CUDA call)
    s->host.resize(s->n_inst);
    std::string err;
    for (int i = 0; i < s->n_inst; ++i) {
        rc = build_instance(*desc, i, &s->host[i], &err);
        if (rc) return fail(rc, err);
        if (s->host[i].ncolours > kMaxColours) return fail(TTS_ERR_UNSUPPORTED, "more than 16 colour classes");
    }
    // nothing from the caller's pointers is kept
    s->desc.pos_explicit = nullptr;
    s->desc.species_explicit = nullptr;
    s->desc.inst_cells = nullptr;
    s->desc.inst_frac1 = nullptr;
    s->desc.inst_peak_Te = nullptr;
    s->desc.inst_fwhm = nullptr;
    s->desc.inst_T_bath = nullptr;
    if (desc->inst_peak_Te) s->inst_peak.assign(desc->inst_peak_Te, desc->inst_peak_Te + s->n_inst);
    if (desc->inst_fwhm) s->inst_fwhm.assign(desc->inst_fwhm, desc->inst_fwhm + s->n_inst);

    // slot layout: instance-major, colour-major inside, ascending atom id
    s->slot_of_atom.resize(s->n_inst);
    s->dinst.resize(s->n_inst);
    int64_t slot = 0;
    int obs_block = 0;
    for (int i = 0; i < s->n_inst; ++i) {
        HostInstance &hi = s->host[i];
        DevInstance &di = s->dinst[i];
        std::memset(&di, 0, sizeof di);
        di.slot_begin = slot;
        di.n = hi.n;
        di.ncolours = hi.ncolours;
        std::vector<int64_t> count(hi.ncolours + 1, 0);
        for (int64_t a = 0; a < hi.n; ++a) count[hi.colour[a] + 1]++;
        for (int c = 0; c < hi.ncolours; ++c) count[c + 1] += count[c];
        for (int c = 0; c <= hi.ncolours; ++c) di.colour_begin[c] = count[c];
        s->slot_of_atom[i].resize(hi.n);
        std::vector<int64_t> next(count.begin(), count.end() - 1);
        for (int64_t a = 0; a < hi.n; ++a) s->slot_of_atom[i][a] = next[hi.colour[a]]++;
        di.cell_begin = i;
        di.ncells = 1;
        di.cells[0] = di.cells[1] = di.cells[2] = 1;
        di.substeps = 1;
        di.sigma_t = 1.0;
        di.obs_block_begin = obs_block;
        di.obs_block_count = static_cast<int>((hi.n + kObsSpan - 1) / kObsSpan);
        obs_block += di.obs_block_count;
        slot += hi.n;
        s->max_colours = std::max(s->max_colours, hi.ncolours);
        for (int64_t a = 0; a < hi.n; ++a)
            s->zmax = std::max<int>(s->zmax, static_cast<int>(hi.nbr_begin[a + 1] - hi.nbr_begin[a]));
    }
    s->n_total = slot;
    s->obs_blocks = obs_block;
    s->max_passes = 2 * s->max_colours - 1;
    if (s->n_total > 0x7fffffffLL) return fail(TTS_ERR_UNSUPPORTED, "more than 2^31 atoms in one system");
    s->merged = false;
    if (s->desc.sweep == TTS_SWEEP_MERGED) {
        // one colour: nothing to merge (the step is a single pass)
        bool same = true;
        for (const HostInstance &hi : s->host) same = same && hi.ncolours == s->host[0].ncolours;
        s->merged = s->max_colours >= 2;
        s->merged_uniform = same;
    }

    // pass ranges: pass p of an instance with K colours takes colour p for
    // p < K-1 (h = dt/2), colour K-1 for p = K-1 (h = dt), colour 2K-2-p after
    s->pass_offset.assign(s->max_passes + 1, 0);
    s->pass_work.assign(s->max_passes, 0);
    for (int pass = 0; pass < s->max_passes; ++pass) {
        s->pass_offset[pass] = static_cast<int64_t>(s->ranges.size());
        int64_t prefix = 0;
        for (int i = 0; i < s->n_inst; ++i) {
            const int K = s->dinst[i].ncolours;
            if (pass >= 2 * K - 1) continue;
            const int c = pass < K - 1 ? pass : (pass == K - 1 ? K - 1 : 2 * K - 2 - pass);
            PassRange r;
            r.slot_begin = s->dinst[i].slot_begin + s->dinst[i].colour_begin[c];
            r.count = s->dinst[i].colour_begin[c + 1] - s->dinst[i].colour_begin[c];
            r.prefix = prefix;
            r.inst = i;
            r.hsel = (pass == K - 1) ? 1 : 0;
            if (r.count == 0) continue;
            prefix += r.count;
            s->ranges.push_back(r);
        }
        s->pass_work[pass] = prefix;
    }
    s->pass_offset[s->max_passes] = static_cast<int64_t>(s->ranges.size());

    // step parameters
    StepParams &p = s->p;
    std::memset(&p, 0, sizeof p);
    for (int t = 0; t < desc->nspecies; ++t) {
        SpeciesParams &sp = p.sp[t];
        sp.mu = desc->mu_muB[t] * kBohrMagneton;
        sp.inv_mu = 1.0 / sp.mu;
        sp.K = desc->K[t];
        sp.kappa = 2.0 * desc->K[t] / sp.mu;
        sp.alpha = desc->alpha[t];
        sp.gprime = kGyro / (1.0 + sp.alpha * sp.alpha);
    }
    const double an = std::sqrt(desc->axis[0] * desc->axis[0] + desc->axis[1] * desc->axis[1] + desc->axis[2] * desc->axis[2]);
    for (int k = 0; k < 3; ++k) {
        p.axis[k] = an > 0.0 ? desc->axis[k] / an : 0.0;
        p.B[k] = desc->B[k];
    }
    p.dt = desc->dt;
    for (int t = 0; t < desc->nspecies; ++t)
        for (int hs = 0; hs < 2; ++hs) {
            const SpeciesParams &sp = p.sp[t];
            const double h = hs ? p.dt : 0.5 * p.dt;
            p.sp[t].sig_c[hs] = sp.alpha > 0.0 ? std::sqrt(2.0 * sp.alpha * kBoltzmann / (kGyro * sp.mu * h)) : 0.0;
        }
    p.key0 = static_cast<uint32_t>(desc->seed & 0xffffffffu);
    p.key1 = static_cast<uint32_t>(desc->seed >> 32);
    p.nspecies = desc->nspecies;
    p.n_total = s->n_total;
    p.zmax = s->zmax;
    p.n_instances = s->n_inst;
    p.instance_base = desc->instance_base;
    p.sample_every = desc->sample_every;
    p.obs_capacity = s->obs_capacity;
    p.ncells_total = s->n_inst;
    p.obs_blocks = s->obs_blocks;

    // engine choice
    s->engine = TTS_ENGINE_GENERAL;
    if (desc->engine == TTS_ENGINE_CHECKER || desc->engine == TTS_ENGINE_RESIDENT ||
        desc->engine == TTS_ENGINE_AUTO) {
        const int want = desc->engine;
        int chosen = engine_select(*desc, s->host, want);
        if (chosen < 0) {
            if (want != TTS_ENGINE_AUTO)
                return fail(TTS_ERR_UNSUPPORTED, "the requested engine cannot run this system");
        } else {
            s->engine = chosen;
        }
    }

    TTS_CUDA(cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking), "create capture stream");

    // device buffers common to all engines
    DevBuffers &b = s->b;
    const int64_t N = s->n_total;
    if ((rc = dev_alloc(&b.inst, s->n_inst, "instance table"))) return rc;
    if ((rc = dev_alloc(&b.ranges, s->ranges.size(), "pass ranges"))) return rc;
    if ((rc = dev_alloc(&b.step, 1, "step counter"))) return rc;
    if ((rc = dev_alloc(&b.open, 1, "sweep state"))) return rc;
    if ((rc = dev_alloc(&b.target, 1, "sweep target"))) return rc;
    if ((rc = dev_alloc(&b.health, 1, "health word"))) return rc;
    if ((rc = dev_alloc(&b.src_energy, s->n_inst, "source energy"))) return rc;
    if ((rc = dev_alloc(&b.obs_partial, size_t(s->obs_blocks) * kObsFields, "observable partials"))) return rc;
    if ((rc = dev_alloc(&b.obs_block_inst, s->obs_blocks, "observable blocks"))) return rc;
    if ((rc = dev_alloc(&b.obs_block_begin, s->obs_blocks, "observable blocks"))) return rc;
    if ((rc = dev_alloc(&b.obs_ring, size_t(s->n_inst) * s->obs_capacity * TTS_NOBS, "observable ring"))) return rc;
    if ((rc = dev_alloc(&b.obs_count, s->n_inst, "observable counts"))) return rc;
    if ((rc = dev_alloc(&b.obs_now, size_t(s->n_inst) * TTS_NOBS, "observable scratch"))) return rc;
    char *q;
    for (void **slotp : {&b.sx, &b.sy, &b.sz}) {
        if ((rc = dev_alloc(&q, N * s->rsize, "spins"))) return rc;
        *slotp = q;
    }
    if ((rc = dev_alloc(&b.atom, N, "atom ids"))) return rc;
    if ((rc = dev_alloc(&b.species, N, "species"))) return rc;
    if ((rc = dev_alloc(&b.cell, N, "cells"))) return rc;
    // the neighbour table also serves the observable kernels of every engine
    if ((rc = dev_alloc(&b.nbr, size_t(s->zmax) * N, "neighbour table"))) return rc;
    if ((rc = dev_alloc(&q, size_t(s->zmax) * N * s->rsize, "coupling table"))) return rc;
    b.nbr_w = q;
    if ((rc = alloc_cells(s.get(), s->n_inst))) return rc;

    // uploads
    rc = s->precision == 64 ? upload_general<double>(s.get()) : upload_general<float>(s.get());
    if (rc) return rc;
    {
        std::vector<int> bi(s->obs_blocks);
        std::vector<int64_t> bb(s->obs_blocks);
        for (int i = 0; i < s->n_inst; ++i)
            for (int k = 0; k < s->dinst[i].obs_block_count; ++k) {
                bi[s->dinst[i].obs_block_begin + k] = i;
                bb[s->dinst[i].obs_block_begin + k] = s->dinst[i].slot_begin + int64_t(k) * kObsSpan;
            }
        if ((rc = upload(b.obs_block_inst, bi.data(), bi.size() * sizeof(int), s->stream, "upload obs blocks"))) return rc;
        if ((rc = upload(b.obs_block_begin, bb.data(), bb.size() * sizeof(int64_t), s->stream, "upload obs blocks"))) return rc;
    }
    std::vector<double> Tb(s->n_inst, desc->T_bath), ones(s->n_inst, 1.0);
    if (desc->inst_T_bath)
        for (int i = 0; i < s->n_inst; ++i) Tb[i] = desc->inst_T_bath[i];
    if ((rc = upload(b.Te, Tb.data(), Tb.size() * sizeof(double), s->stream, "upload bath"))) return rc;
    if ((rc = upload(b.Tl, Tb.data(), Tb.size() * sizeof(double), s->stream, "upload bath"))) return rc;
    if ((rc = upload(b.src_shape, ones.data(), ones.size() * sizeof(double), s->stream, "upload shape"))) return rc;
    if ((rc = upload(b.inst, s->dinst.data(), s->dinst.size() * sizeof(DevInstance), s->stream, "upload instances"))) return rc;
    if ((rc = upload(b.ranges, s->ranges.data(), s->ranges.size() * sizeof(PassRange), s->stream, "upload ranges"))) return rc;
    TTS_CUDA(cudaMemsetAsync(b.step, 0, sizeof(int64_t), s->stream), "zero step");
    TTS_CUDA(cudaMemsetAsync(b.open, 0, sizeof(int), s->stream), "zero sweep state");
    TTS_CUDA(cudaMemsetAsync(b.target, 0, sizeof(int64_t), s->stream), "zero sweep target");
    TTS_CUDA(cudaMemsetAsync(b.health, 0, sizeof(unsigned), s->stream), "zero health");
    TTS_CUDA(cudaMemsetAsync(b.src_energy, 0, s->n_inst * sizeof(double), s->stream), "zero energy");
    TTS_CUDA(cudaMemsetAsync(b.obs_count, 0, s->n_inst * sizeof(int64_t), s->stream), "zero obs");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "create");

    if (s->engine != TTS_ENGINE_GENERAL) {
        rc = engine_create(*desc, s->host, s->slot_of_atom, s->dinst, s->p, s->b, s->engine, s->stream, &s->eng);
        if (rc) return fail(rc, std::string("engine set-up failed: ") + engine_last_error());
    }
    s->p.sigma_per_step = 0;                 // uniform bath: the table never changes
    if ((rc = refresh_sigma(s.get()))) return rc;
    *out = s.release();
    return TTS_OK;
}

int tts_set_ttm_grid(tts_system *s, const tts_ttm_desc *t)
{
    if (!s || !t) return fail(TTS_ERR_ARG, "null argument");
    if (s->desc.lattice == TTS_LATTICE_CLUSTER) return fail(TTS_ERR_UNSUPPORTED, "TTM grids need a periodic lattice");
    for (int k = 0; k < 3; ++k)
        if (t->cells[k] < 1) return fail(TTS_ERR_ARG, "TTM cell counts must be >= 1");
    if (!(t->gamma_e > 0.0) || !(t->C_l > 0.0) || !(t->G >= 0.0) || !(t->kappa_e >= 0.0) || !(t->T0 > 0.0))
        return fail(TTS_ERR_ARG, "TTM coefficients out of range");
    if (t->source < 0 || t->source > 3 || t->spatial < 0 || t->spatial > 2) return fail(TTS_ERR_ARG, "bad TTM mode");
    const bool profile = t->source == TTS_SOURCE_STEP_PROFILE;
    if (profile && s->lat) return fail(TTS_ERR_UNSUPPORTED, "the step profile is for rigid lattices");
    if (profile && !(t->t0 >= 0.0)) return fail(TTS_ERR_ARG, "step profile: t0 (first stage) must be >= 0");
    if (t->spatial == TTS_SPATIAL_XY_GAUSS && !(t->sigma_xy > 0.0))
        return fail(TTS_ERR_ARG, "the Gaussian spot needs sigma_xy > 0");
    if (t->spatial == TTS_SPATIAL_Z_EXP && !(t->depth_z > 0.0))
        return fail(TTS_ERR_ARG, "the exponential profile needs depth_z > 0");
    {
        // cells over all instances must fit the int indices of the grid kernels
        int64_t cells = s->n_inst;
        for (int k = 0; k < 3; ++k) {
            if (t->cells[k] > INT_MAX / cells) return fail(TTS_ERR_ARG, "TTM grid too large");
            cells *= t->cells[k];
        }
    }
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set ttm");
    const int nc = t->cells[0] * t->cells[1] * t->cells[2];
    const int total = nc * s->n_inst;
    int rc = alloc_cells(s, total);
    if (rc) return rc;
    std::vector<double> shape(total), Te(total, t->T0);
    std::vector<int> cellmap(s->n_total);
    s->P0.assign(s->n_inst, t->P0);
    // calibration jobs: one per distinct (box, peak, pulse width); the jobs run
    // on the GPU, one CTA each
    struct CalKey { double box[3], peak, fwhm; };
    std::vector<CalKey> keys;
    std::vector<int> job_of(s->n_inst, -1);
    std::vector<HostTtm> hts(s->n_inst);
    for (int i = 0; i < s->n_inst; ++i) {
        const HostInstance &hi = s->host[i];
        DevInstance &di = s->dinst[i];
        const double my_fwhm = s->inst_fwhm.empty() ? t->fwhm : s->inst_fwhm[i];
        const double my_peak = s->inst_peak.empty() ? t->peak_Te : s->inst_peak[i];
        if (profile && !(my_fwhm >= 0.0 && my_peak >= 0.0))
            return fail(TTS_ERR_ARG, "step profile: peak and second-stage duration must be >= 0");
        if (!profile && t->source != TTS_SOURCE_NONE && !(my_fwhm > 0.0)) return fail(TTS_ERR_ARG, "pulse FWHM must be positive");
        HostTtm &h = hts[i];
        make_host_ttm(lattice_step_length(s), hi, *t, t->source != TTS_SOURCE_NONE && !profile ? my_fwhm : 1.0, &h);
        if (t->source == TTS_SOURCE_PEAK) {
            if (!(my_peak > t->T0)) return fail(TTS_ERR_ARG, "peak T_e must exceed T0");
            // a one-cell grid has no length scale: its calibration ignores the box
            const double kb[3] = {nc > 1 ? hi.box[0] : 0.0, nc > 1 ? hi.box[1] : 0.0, nc > 1 ? hi.box[2] : 0.0};
            for (size_t k = 0; k < keys.size(); ++k)
                if (keys[k].box[0] == kb[0] && keys[k].box[1] == kb[1] && keys[k].box[2] == kb[2] &&
                    keys[k].peak == my_peak && keys[k].fwhm == my_fwhm)
                    job_of[i] = static_cast<int>(k);
            if (job_of[i] < 0) {
                job_of[i] = static_cast<int>(keys.size());
                keys.push_back({{kb[0], kb[1], kb[2]}, my_peak, my_fwhm});
            }
        }
        di.cell_begin = i * nc;
        di.ncells = nc;
        for (int k = 0; k < 3; ++k) {
            di.cells[k] = t->cells[k];
            di.dx[k] = h.dx[k];
            di.inv_dx2[k] = 1.0 / (h.dx[k] * h.dx[k]);
        }
        di.cell_volume = h.vol;
        di.substeps = profile ? 1 : h.substeps;
        di.prof_peak = my_peak;
        di.prof_t1 = t->t0;
        di.prof_t2 = t->t0 + my_fwhm;
        di.P0 = t->P0;
        di.sigma_t = h.sigma_t;
        di.t0 = h.t0;
        for (int c = 0; c < nc; ++c) shape[di.cell_begin + c] = h.shape[c];
        // cell of each atom: floor(x / L * n) on the exact half-lattice coordinate
        for (int64_t a = 0; a < hi.n; ++a) {
            int cc[3];
            for (int k = 0; k < 3; ++k)
                cc[k] = static_cast<int>((int64_t(hi.half[3 * a + k]) * t->cells[k]) / (2LL * hi.cells[k]));
            cellmap[di.slot_begin + s->slot_of_atom[i][a]] = di.cell_begin + (cc[2] * t->cells[1] + cc[1]) * t->cells[0] + cc[0];
        }
    }
    TtmParams tp{};
    tp.active = 1;
    tp.gamma_e = t->gamma_e;
    tp.C_l = t->C_l;
    tp.inv_gamma_e = 1.0 / t->gamma_e;
    tp.inv_C_l = 1.0 / t->C_l;
    tp.G = t->G;
    tp.kappa_e = t->kappa_e;
    tp.T0 = t->T0;
    tp.source = t->source;
    tp.spatial = t->spatial;
    tp.sigma_xy = t->sigma_xy;
    tp.depth_z = t->depth_z;
    if (!keys.empty()) {
        const int nj = static_cast<int>(keys.size());
        const int NC = 32;                       // candidate powers per job and round
        std::vector<int> first(nj, -1);
        for (int i = 0; i < s->n_inst; ++i)
            if (job_of[i] >= 0 && first[job_of[i]] < 0) first[job_of[i]] = i;
        std::vector<CalibJob> jobs(nj);
        double *shape_dev = nullptr, *work_dev = nullptr, *cand_dev = nullptr, *peak_dev = nullptr;
        CalibJob *jobs_dev = nullptr;
        auto release = [&]() {
            cudaFree(shape_dev);
            cudaFree(work_dev);
            cudaFree(jobs_dev);
            cudaFree(cand_dev);
            cudaFree(peak_dev);
        };
        if ((rc = dev_alloc(&shape_dev, size_t(nj) * nc, "calibration shapes")) ||
            (rc = dev_alloc(&work_dev, size_t(nj) * NC * 3 * nc, "calibration scratch")) ||
            (rc = dev_alloc(&jobs_dev, nj, "calibration jobs")) ||
            (rc = dev_alloc(&cand_dev, size_t(nj) * NC, "calibration candidates")) ||
            (rc = dev_alloc(&peak_dev, size_t(nj) * NC, "calibration peaks"))) {
            release();
            return rc;
        }
        std::vector<double> lo(nj, 0.0), hi(nj, 0.0), guess(nj), cand(size_t(nj) * NC), peaks(size_t(nj) * NC);
        std::vector<int> bracketed(nj, 0);
        for (int j = 0; j < nj; ++j) {
            const HostTtm &h = hts[first[j]];
            CalibJob &J = jobs[j];
            std::memset(&J, 0, sizeof J);
            for (int k = 0; k < 3; ++k) {
                J.cells[k] = h.cells[k];
                J.dx[k] = h.dx[k];
            }
            J.substeps = h.substeps;
            J.sigma_t = h.sigma_t;
            J.t0 = h.t0;
            J.nsteps = static_cast<int64_t>(std::ceil((h.t0 + 10.0 * h.sigma_t) / lattice_step_length(s)));
            J.shape = shape_dev + size_t(j) * nc;
            J.work = work_dev + size_t(j) * NC * 3 * nc;
            guess[j] = 0.5 * t->gamma_e * (keys[j].peak * keys[j].peak - t->T0 * t->T0) /
                       (h.sigma_t * std::sqrt(2.0 * M_PI));
            cudaMemcpyAsync(shape_dev + size_t(j) * nc, h.shape.data(), nc * sizeof(double), cudaMemcpyHostToDevice,
                            s->stream);
        }
        cudaMemcpyAsync(jobs_dev, jobs.data(), nj * sizeof(CalibJob), cudaMemcpyHostToDevice, s->stream);
        cudaError_t e = cudaSuccess;
        auto evaluate = [&]() {
            e = cudaMemcpyAsync(cand_dev, cand.data(), cand.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = launch_calibrate(jobs_dev, cand_dev, peak_dev, nj, NC, nc, lattice_step_length(s), tp, s->stream);
            ++s->launches;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(peaks.data(), peak_dev, peaks.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        };
        // bracket: powers guess * 2^c; the peak grows without bound with P0
        for (int round = 0; round < 8 && e == cudaSuccess; ++round) {
            bool all = true;
            for (int j = 0; j < nj; ++j) {
                all = all && bracketed[j];
                for (int c = 0; c < NC; ++c) cand[j * NC + c] = guess[j] * std::ldexp(1.0, c);
            }
            if (all) break;
            evaluate();
            for (int j = 0; j < nj && e == cudaSuccess; ++j) {
                if (bracketed[j]) continue;
                for (int c = 0; c < NC; ++c)
                    if (peaks[j * NC + c] >= keys[j].peak) {
                        hi[j] = cand[j * NC + c];
                        lo[j] = c > 0 ? cand[j * NC + c - 1] : 0.0;
                        bracketed[j] = 1;
                        break;
                    }
                if (!bracketed[j]) guess[j] = cand[j * NC + NC - 1] * 2.0;
            }
        }
        for (int j = 0; j < nj && e == cudaSuccess; ++j)
            if (!bracketed[j]) e = cudaErrorInvalidValue;
        // multi-section: each round splits [lo, hi] into NC + 1 parts
        for (int round = 0; round < 14 && e == cudaSuccess; ++round) {
            bool done = true;
            for (int j = 0; j < nj; ++j) {
                done = done && (hi[j] - lo[j]) <= 4e-16 * hi[j];   // a few ulps of hi
                for (int c = 0; c < NC; ++c) cand[j * NC + c] = lo[j] + (hi[j] - lo[j]) * (c + 1) / (NC + 1);
            }
            if (done) break;
            evaluate();
            for (int j = 0; j < nj && e == cudaSuccess; ++j) {
                int c = 0;
                while (c < NC && peaks[j * NC + c] < keys[j].peak) ++c;
                const double new_lo = c > 0 ? cand[j * NC + c - 1] : lo[j];
                const double new_hi = c < NC ? cand[j * NC + c] : hi[j];
                lo[j] = new_lo;
                hi[j] = new_hi;
            }
        }
        release();
        if (e != cudaSuccess) return cuda_fail(e, "source calibration");
        for (int i = 0; i < s->n_inst; ++i)
            if (job_of[i] >= 0) {
                s->P0[i] = 0.5 * (lo[job_of[i]] + hi[job_of[i]]);
                s->dinst[i].P0 = s->P0[i];
            }
    }
    DevBuffers &b = s->b;
    {
        std::vector<int> ci(total);
        bool one = true;
        for (int i = 0; i < s->n_inst; ++i) {
            for (int c = 0; c < nc; ++c) ci[i * nc + c] = i;
            one = one && s->dinst[i].substeps == 1;
        }
        if ((rc = upload(b.cell_inst, ci.data(), ci.size() * sizeof(int), s->stream, "upload cell instances"))) return rc;
        s->p.ttm_one_substep = one && !s->lat ? 1 : 0;
    }
    std::vector<double> Tl0(Te);
    if (profile) {
        // the profile at the current time
        int64_t step = 0;
        TTS_CUDA(cudaMemcpy(&step, b.step, sizeof step, cudaMemcpyDeviceToHost), "read step");
        const double tt = double(step) * s->desc.dt;
        for (int i = 0; i < s->n_inst; ++i) {
            const DevInstance &di = s->dinst[i];
            const double T = tt < di.prof_t1 ? di.prof_peak : (tt < di.prof_t2 ? 0.5 * di.prof_peak : t->T0);
            for (int c = 0; c < nc; ++c) Te[i * nc + c] = T;
        }
    }
    if ((rc = upload(b.Te, Te.data(), total * sizeof(double), s->stream, "upload T_e"))) return rc;
    if ((rc = upload(b.Tl, Tl0.data(), total * sizeof(double), s->stream, "upload T_l"))) return rc;
    if ((rc = upload(b.src_shape, shape.data(), total * sizeof(double), s->stream, "upload shape"))) return rc;
    if ((rc = upload(b.cell, cellmap.data(), cellmap.size() * sizeof(int), s->stream, "upload cell map"))) return rc;
    if ((rc = upload(b.inst, s->dinst.data(), s->dinst.size() * sizeof(DevInstance), s->stream, "upload instances"))) return rc;
    TTS_CUDA(cudaMemsetAsync(b.src_energy, 0, s->n_inst * sizeof(double), s->stream), "zero energy");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set ttm");
    s->tp = tp;
    s->ttm_active = true;
    s->p.sigma_per_step = s->p.ttm_one_substep ? 0 : 1;
    if ((rc = refresh_sigma(s))) return rc;
    if (s->lat) {
        // bath cells from the current positions; ion energy tallies per cell
        if ((rc = lattice_ensure_cell_acc(s)) || (rc = lattice_refresh_now(s))) return rc;
    }
    if (s->eng) {
        rc = engine_set_cells(s->eng, s->dinst, cellmap, s->stream);
        if (rc) {
            if (s->desc.engine != TTS_ENGINE_AUTO)
                return fail(rc, std::string("engine TTM set-up failed: ") + engine_last_error());
            // AUTO: the general arrays hold the spins of a resident system, so
            // the next valid engine can take over directly
            engine_destroy(s->eng);
            s->eng = nullptr;
            s->engine = TTS_ENGINE_GENERAL;
            if (engine_select(s->desc, s->host, TTS_ENGINE_CHECKER) == TTS_ENGINE_CHECKER &&
                engine_create(s->desc, s->host, s->slot_of_atom, s->dinst, s->p, s->b, TTS_ENGINE_CHECKER, s->stream,
                              &s->eng) == TTS_OK)
                s->engine = TTS_ENGINE_CHECKER;
        }
    }
    s->dirty = true;
    return TTS_OK;
}

int tts_step(tts_system *s, int64_t nsteps)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    if (nsteps < 0) return fail(TTS_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return TTS_OK;
    if (s->merged && !s->eng && !s->merged_uniform)
        return fail(TTS_ERR_UNSUPPORTED, "the merged sweep on the general engine needs the same colour count in every instance");
    // every path below advances the device counter by nsteps
    const int64_t step0 = s->host_step;
    s->host_step += nsteps;
    if (s->merged && !(s->eng && engine_multi_step(s->eng))) {
        // the last step of this call closes the merged sweep
        TTS_CUDA(launch_set_target(s->b, nsteps, s->stream), "sweep target");
        s->launches += 1;
    }
    if (s->eng && engine_multi_step(s->eng)) {
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (s->profiling) {
            TTS_CUDA(cudaEventCreate(&ev[0]), "profile event");
            TTS_CUDA(cudaEventCreate(&ev[1]), "profile event");
            s->prof_events.push_back(ev[0]);
            s->prof_events.push_back(ev[1]);
            s->prof_pair_steps.push_back(nsteps);
        }
        int kernels = 0;
        StepParams p = s->p;
        p.merged = s->merged ? 1 : 0;
        cudaError_t e = engine_run_steps(s->eng, p, s->b, s->tp, s->ttm_active, nsteps, s->stream, &kernels,
                                         ev[0], ev[1]);
        if (e != cudaSuccess) return cuda_fail(e, "resident steps");
        s->launches += kernels;
        return TTS_OK;
    }
    if (s->profiling) {
        // The steps, with timing events around their colour passes, are
        // captured into one graph and replayed: the device runs them back to
        // back as in the timed path, instead of waiting on the host's launches
        // between kernels.  Every kernel is a node of its own (no step graph
        // is reused), so the launch count stays exact.
        cudaStream_t c = s->capture;
        TTS_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "begin profiled capture");
        cudaError_t e = cudaSuccess;
        int total = 0;
        for (int64_t i = 0; i < nsteps && e == cudaSuccess; ++i) {
            cudaEvent_t ev[2] = {nullptr, nullptr};
            e = cudaEventCreate(&ev[0]);
            if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
            if (ev[0]) s->prof_events.push_back(ev[0]);
            if (ev[1]) s->prof_events.push_back(ev[1]);
            if (e != cudaSuccess) break;
            s->prof_pair_steps.push_back(1);
            int kernels = 0;
            e = record_step(s, c, &kernels, ev[0], ev[1], true, step0 + i);
            total += kernels;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c, &g);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t x = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = cudaGraphLaunch(x, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // before the executable graph goes
        if (x) cudaGraphExecDestroy(x);
        if (e != cudaSuccess) {
            drop_profile_events(s);
            return cuda_fail(e, "profiled steps");
        }
        s->launches += total;
        return TTS_OK;
    }
    if (s->dirty) {
        int rc = build_graph(s);
        if (rc) return rc;
    }
    // the graph variant of the parity of the step it starts at
    int64_t at = step0;
    auto var = [&]() { return s->by_parity ? static_cast<int>(at & 1) : 0; };
    if (!s->phased) {
        int64_t left = nsteps;
        for (; left >= s->graph_steps; left -= s->graph_steps, at += s->graph_steps) {
            TTS_CUDA(cudaGraphLaunch(s->graph_multi[var()], s->stream), "launch step graph");
            s->launches += s->kernels_multi;
        }
        for (; left > 0; --left, ++at) {
            TTS_CUDA(cudaGraphLaunch(s->graph[var()], s->stream), "launch step graph");
            s->launches += s->kernels_graph;
        }
        return TTS_OK;
    }
    cudaError_t err = cudaSuccess;
    schedule_steps(step0, nsteps, s->p.sample_every, s->graph_steps, s->cycle_steps, [&](StepGraph g, int64_t n) {
        if (err != cudaSuccess) return;
        const int v = var();
        at += n;
        cudaGraphExec_t x = s->graph[v];
        int k = s->kernels_graph;
        if (g == StepGraph::Cycle) {
            x = s->graph_cycle[v];
            k = s->kernels_cycle;
        } else if (g == StepGraph::PlainRun) {
            x = s->graph_multi[v];
            k = s->kernels_multi;
        } else if (g == StepGraph::Plain) {
            x = s->graph_plain[v];
            k = s->kernels_plain;
        }
        err = cudaGraphLaunch(x, s->stream);
        if (err == cudaSuccess) s->launches += k;
    });
    if (err != cudaSuccess) return cuda_fail(err, "launch step graph");
    return TTS_OK;
}

int tts_autotune(tts_system *s, int probe_steps, int *chosen, int *n_configs)
{
    if (!s || probe_steps < 1) return fail(TTS_ERR_ARG, "bad argument");
    if (s->profiling) return fail(TTS_ERR_STATE, "switch profiling off before autotuning");
    const int n = s->eng ? engine_num_configs(s->eng) : static_cast<int>(s->pass_blocks.size());
    if (n_configs) *n_configs = n;
    if (n <= 1) {
        if (chosen) *chosen = 0;
        return TTS_OK;
    }
    // cache key: engine, precision, instance count and every instance's shape
    std::string key = std::to_string(s->engine) + "/" + std::to_string(s->precision) + "/" +
                      std::to_string(s->n_inst) + "/" + std::to_string(s->zmax) + "/" + std::to_string(s->lat != nullptr);
    for (const HostInstance &hi : s->host)
        key += ":" + std::to_string(hi.cells[0]) + "x" + std::to_string(hi.cells[1]) + "x" + std::to_string(hi.cells[2]);
    static std::mutex cache_lock;
    static std::map<std::string, int> cache;
    int best = -1;
    {
        std::lock_guard<std::mutex> g(cache_lock);
        auto it = cache.find(key);
        if (it != cache.end()) best = it->second;
    }
    if (best < 0) {
        size_t nbytes = 0;
        int rc = tts_get_state(s, nullptr, &nbytes);
        if (rc) return rc;
        std::vector<char> saved(nbytes);
        if ((rc = tts_get_state(s, saved.data(), &nbytes))) return rc;
        const int64_t launches0 = s->launches;
        cudaEvent_t e0, e1;
        TTS_CUDA(cudaEventCreate(&e0), "autotune event");
        TTS_CUDA(cudaEventCreate(&e1), "autotune event");
        float best_ms = 0.0f;
        for (int c = 0; c < n && !rc; ++c) {
            if (s->eng) engine_set_config(s->eng, c);
            else s->pass_block = s->pass_blocks[c];
            s->dirty = true;
            if ((rc = tts_step(s, 2))) break;                       // graph build and warm-up
            if (cudaEventRecord(e0, s->stream) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "autotune"); break; }
            if ((rc = tts_step(s, probe_steps))) break;
            cudaEventRecord(e1, s->stream);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "autotune"); break; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0 || ms < best_ms) {
                best = c;
                best_ms = ms;
            }
            if ((rc = tts_set_state(s, saved.data(), nbytes))) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        s->launches = launches0;
        std::lock_guard<std::mutex> g(cache_lock);
        cache[key] = best;
    }
    if (s->eng) engine_set_config(s->eng, best);
    else s->pass_block = s->pass_blocks[best];
    s->dirty = true;
    if (chosen) *chosen = best;
    // the chosen configuration may read the other noise table: both from T_e
    return refresh_sigma(s);
}

int tts_set_config(tts_system *s, int index, int *current, int *n_configs)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    const int n = s->eng ? engine_num_configs(s->eng) : static_cast<int>(s->pass_blocks.size());
    if (n_configs) *n_configs = n;
    if (index >= n) return fail(TTS_ERR_ARG, "configuration index out of range");
    if (index >= 0 && n > 0) {
        if (s->eng) engine_set_config(s->eng, index);
        else s->pass_block = s->pass_blocks[index];
        s->dirty = true;
        // a configuration may read the other noise table: both from T_e
        int rc = refresh_sigma(s);
        if (rc) return rc;
    }
    if (current) {
        if (s->eng) *current = engine_config(s->eng);
        else {
            int c = 0;
            for (int k = 0; k < n; ++k)
                if (s->pass_blocks[k] == s->pass_block) c = k;
            *current = c;
        }
    }
    return TTS_OK;
}

int tts_profile_enable(tts_system *s, int enable)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "profile enable");
    drop_profile_events(s);
    s->prof_ms = 0.0;
    s->prof_steps = 0;
    s->profiling = enable != 0;
    // profiled steps keep the TTM after the passes and one noise table: both
    // tables from T_e, whichever the next step reads
    return refresh_sigma(s);
}

int tts_profile_read(tts_system *s, double *ms, int64_t *steps, int64_t *spin_steps)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "profile read");
    for (size_t k = 0; k + 1 < s->prof_events.size(); k += 2) {
        float t = 0.0f;
        TTS_CUDA(cudaEventElapsedTime(&t, s->prof_events[k], s->prof_events[k + 1]), "profile elapsed");
        s->prof_ms += t;
        s->prof_steps += s->prof_pair_steps[k / 2];
    }
    drop_profile_events(s);
    if (ms) *ms = s->prof_ms;
    if (steps) *steps = s->prof_steps;
    if (spin_steps) *spin_steps = s->prof_steps * lattice_units_per_step(s);
    return TTS_OK;
}

int tts_sync(tts_system *s)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "synchronise");
    unsigned h = 0;
    TTS_CUDA(cudaMemcpy(&h, s->b.health, sizeof h, cudaMemcpyDeviceToHost), "read health");
    if (h & kHealthTimeout) return fail(TTS_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    if (h & kHealthNonFinite) return fail(TTS_ERR_HEALTH, "non-finite spin produced on the device");
    if (h & kHealthSkin) return fail(TTS_ERR_HEALTH, "an atom moved further than half the skin from its site");
    if (h & kHealthColour) return fail(TTS_ERR_HEALTH, "two exchange-coupled atoms share a colour class");
    if (h & kHealthOverflow) return fail(TTS_ERR_HEALTH, "more exchange neighbours than the table holds");
    return TTS_OK;
}

int tts_observables(tts_system *s, int inst, double *out, int64_t max_samples, int64_t *n_written)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!out || !n_written || max_samples < 0) return fail(TTS_ERR_ARG, "bad output arguments");
    if ((rc = tts_sync(s))) return rc;
    int64_t count = 0;
    TTS_CUDA(cudaMemcpy(&count, s->b.obs_count + inst, sizeof count, cudaMemcpyDeviceToHost), "read obs count");
    const int64_t cap = s->obs_capacity;
    const int64_t have = std::min(count, cap);
    std::vector<double> ring(size_t(cap) * TTS_NOBS);
    TTS_CUDA(cudaMemcpy(ring.data(), s->b.obs_ring + size_t(inst) * cap * TTS_NOBS, ring.size() * sizeof(double),
                        cudaMemcpyDeviceToHost), "read obs ring");
    const int64_t first = count - have;
    const int64_t m = std::min(have, max_samples);
    for (int64_t k = 0; k < m; ++k) {
        const int64_t src = (first + k) % cap;
        std::memcpy(out + k * TTS_NOBS, ring.data() + src * TTS_NOBS, TTS_NOBS * sizeof(double));
    }
    *n_written = m;
    return TTS_OK;
}

int tts_observe_now(tts_system *s, int inst, double *out)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!out) return fail(TTS_ERR_ARG, "null output");
    cudaError_t e = cudaErrorNotSupported;
    if (s->eng) {
        StepParams p = s->p;
        p.obs_blocks = s->obs_blocks;
        e = engine_obs_partials(s->eng, p, s->b, 1, s->stream);
        if (e == cudaSuccess) {
            e = launch_obs_reduce(p, s->b, 1, s->stream);
            s->launches += 2;
            if (e != cudaSuccess) return cuda_fail(e, "observe");
        } else if (e != cudaErrorNotSupported) {
            return cuda_fail(e, "observe");
        } else {
            e = engine_sync_to_general(s->eng, s->b, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "engine gather");
            e = cudaErrorNotSupported;
        }
    }
    if (e == cudaErrorNotSupported) {
        e = launch_obs(s->p, s->b, s->precision, s->obs_blocks, 1, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "observe");
        s->launches += 2;
    }
    TTS_CUDA(cudaStreamSynchronize(s->stream), "observe");
    TTS_CUDA(cudaMemcpy(out, s->b.obs_now + size_t(inst) * TTS_NOBS, TTS_NOBS * sizeof(double), cudaMemcpyDeviceToHost),
             "read observation");
    return TTS_OK;
}

int tts_get_spins(tts_system *s, int inst, double *xyz)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!xyz) return fail(TTS_ERR_ARG, "null output");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get spins");
    return s->precision == 64 ? read_instance_spins<double>(s, inst, xyz) : read_instance_spins<float>(s, inst, xyz);
}

int tts_set_spins(tts_system *s, int inst, const double *xyz)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!xyz) return fail(TTS_ERR_ARG, "null input");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set spins");
    return s->precision == 64 ? write_instance_spins<double>(s, inst, xyz) : write_instance_spins<float>(s, inst, xyz);
}

int tts_get_all_spins(tts_system *s, double *xyz)
{
    if (!s || !xyz) return fail(TTS_ERR_ARG, "null argument");
    for (int i = 0; i < s->n_inst; ++i) {
        int rc = tts_get_spins(s, i, xyz);
        if (rc) return rc;
        xyz += 3 * s->dinst[i].n;
    }
    return TTS_OK;
}

int tts_set_all_spins(tts_system *s, const double *xyz)
{
    if (!s || !xyz) return fail(TTS_ERR_ARG, "null argument");
    for (int i = 0; i < s->n_inst; ++i) {
        int rc = tts_set_spins(s, i, xyz);
        if (rc) return rc;
        xyz += 3 * s->dinst[i].n;
    }
    return TTS_OK;
}

namespace {
int io_buffer(tts_system *s)
{
    if (s->io_buf) return TTS_OK;
    cudaError_t e = cudaMalloc(&s->io_buf, size_t(s->n_total) * 3 * s->rsize);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->io_buf = nullptr;
        return fail(TTS_ERR_OOM, "spin I/O staging buffer");
    }
    return TTS_OK;
}
}  // namespace

int tts_read_spins_async(tts_system *s, void *host, size_t bytes)
{
    if (!s || !host) return fail(TTS_ERR_ARG, "null argument");
    if (bytes != size_t(s->n_total) * 3 * s->rsize) return fail(TTS_ERR_ARG, "byte count is not 3 n_total reals");
    int rc = io_buffer(s);
    if (rc) return rc;
    if (s->eng) {
        cudaError_t e = engine_sync_to_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine gather");
    }
    TTS_CUDA(launch_spins_to_atoms(s->b, s->n_total, s->n_inst, s->precision, s->io_buf, s->stream), "spin reorder");
    TTS_CUDA(cudaMemcpyAsync(host, s->io_buf, bytes, cudaMemcpyDeviceToHost, s->stream), "read spins");
    s->launches += s->eng ? 2 : 1;
    return TTS_OK;
}

int tts_write_spins_async(tts_system *s, const void *host, size_t bytes)
{
    if (!s || !host) return fail(TTS_ERR_ARG, "null argument");
    if (bytes != size_t(s->n_total) * 3 * s->rsize) return fail(TTS_ERR_ARG, "byte count is not 3 n_total reals");
    int rc = io_buffer(s);
    if (rc) return rc;
    TTS_CUDA(cudaMemcpyAsync(s->io_buf, host, bytes, cudaMemcpyHostToDevice, s->stream), "write spins");
    TTS_CUDA(launch_spins_from_atoms(s->b, s->n_total, s->n_inst, s->precision, s->io_buf, s->stream), "spin reorder");
    if (s->eng) {
        cudaError_t e = engine_sync_from_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine scatter");
    }
    s->launches += s->eng ? 2 : 1;
    return TTS_OK;
}

int tts_instance_size(tts_system *s, int inst, int64_t *n, int *ncol)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (n) *n = s->dinst[inst].n;
    if (ncol) *ncol = s->dinst[inst].ncolours;
    return TTS_OK;
}

int tts_get_species(tts_system *s, int inst, int *out)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!out) return fail(TTS_ERR_ARG, "null output");
    for (int64_t a = 0; a < s->dinst[inst].n; ++a) out[a] = s->host[inst].species[a];
    return TTS_OK;
}

int tts_get_colours(tts_system *s, int inst, int *out)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!out) return fail(TTS_ERR_ARG, "null output");
    for (int64_t a = 0; a < s->dinst[inst].n; ++a) out[a] = s->host[inst].colour[a];
    return TTS_OK;
}

int tts_get_ttm(tts_system *s, int inst, double *Te, double *Tl, double *P0)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get ttm");
    const DevInstance &di = s->dinst[inst];
    if (Te) TTS_CUDA(cudaMemcpy(Te, s->b.Te + di.cell_begin, di.ncells * sizeof(double), cudaMemcpyDeviceToHost), "read T_e");
    if (Tl) TTS_CUDA(cudaMemcpy(Tl, s->b.Tl + di.cell_begin, di.ncells * sizeof(double), cudaMemcpyDeviceToHost), "read T_l");
    if (P0) *P0 = s->ttm_active ? s->P0[inst] : 0.0;
    return TTS_OK;
}

int tts_set_ttm_state(tts_system *s, int inst, const double *Te, const double *Tl)
{
    int rc = check_inst(s, inst);
    if (rc) return rc;
    if (!s->ttm_active) return fail(TTS_ERR_STATE, "no TTM grid set");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set ttm state");
    const DevInstance &di = s->dinst[inst];
    if (Te) TTS_CUDA(cudaMemcpy(s->b.Te + di.cell_begin, Te, di.ncells * sizeof(double), cudaMemcpyHostToDevice), "write T_e");
    if (Tl) TTS_CUDA(cudaMemcpy(s->b.Tl + di.cell_begin, Tl, di.ncells * sizeof(double), cudaMemcpyHostToDevice), "write T_l");
    return refresh_sigma(s);
}

int tts_get_step(tts_system *s, int64_t *step)
{
    if (!s || !step) return fail(TTS_ERR_ARG, "null argument");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get step");
    TTS_CUDA(cudaMemcpy(step, s->b.step, sizeof(int64_t), cudaMemcpyDeviceToHost), "read step");
    return TTS_OK;
}

int tts_set_step(tts_system *s, int64_t step)
{
    if (!s || step < 0) return fail(TTS_ERR_ARG, "bad argument");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set step");
    TTS_CUDA(cudaMemcpy(s->b.step, &step, sizeof(int64_t), cudaMemcpyHostToDevice), "write step");
    TTS_CUDA(cudaMemset(s->b.open, 0, sizeof(int)), "reset sweep state");
    s->host_step = step;
    return refresh_sigma(s);     // the table a pass reads may depend on the step's parity
}

static_assert(kHealthNonFinite == TTS_HEALTH_NONFINITE && kHealthTimeout == TTS_HEALTH_TIMEOUT &&
                  kHealthSkin == TTS_HEALTH_SKIN && kHealthColour == TTS_HEALTH_COLOUR &&
                  kHealthOverflow == TTS_HEALTH_OVERFLOW,
              "device health bits and their ABI values");

int tts_health(tts_system *s, unsigned *bits)
{
    if (!s || !bits) return fail(TTS_ERR_ARG, "null argument");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "synchronise");
    TTS_CUDA(cudaMemcpy(bits, s->b.health, sizeof(unsigned), cudaMemcpyDeviceToHost), "read health");
    return TTS_OK;
}

namespace {
// A wait that no transfer completes: the barrier expects 16 bytes that are
// never sent, so the bounded wait runs out and the kernel reports it.
__global__ void selftest_wait_kernel(unsigned *health, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_init_fence();
    mbar_arrive_expect_tx(&bar, 16u);
    if (!mbar_wait(&bar, 0u, limit_ns)) atomicOr(health, kHealthTimeout);
}
}  // namespace

int tts_selftest_wait(tts_system *s, int64_t limit_ns)
{
    if (!s) return fail(TTS_ERR_ARG, "null system");
    if (!(limit_ns > 0 && limit_ns <= 10000000000ll)) return fail(TTS_ERR_ARG, "limit must be in (0, 10 s]");
    selftest_wait_kernel<<<1, 32, 0, s->stream>>>(s->b.health, static_cast<uint64_t>(limit_ns));
    ++s->launches;
    TTS_CUDA(cudaGetLastError(), "self-test launch");
    return TTS_OK;
}

int tts_info(tts_system *s, tts_info_t *info)
{
    if (!s || !info) return fail(TTS_ERR_ARG, "null argument");
    info->n_total = s->n_total;
    info->n_instances = s->n_inst;
    info->engine = s->engine;
    info->precision = s->precision;
    info->max_colours = s->max_colours;
    int64_t st = 0;
    TTS_CUDA(cudaStreamSynchronize(s->stream), "info");
    TTS_CUDA(cudaMemcpy(&st, s->b.step, sizeof st, cudaMemcpyDeviceToHost), "read step");
    info->steps_done = st;
    info->kernel_launches = s->launches;
    return TTS_OK;
}

// Checkpoint layout: header {magic, version, precision, n_total, n_inst,
// ncells_total, obs_capacity}, step, then spins (slot order, 3 arrays),
// T_e, T_l, source energies, observable counts and rings.
int tts_get_state(tts_system *s, void *buf, size_t *nbytes)
{
    if (!s || !nbytes) return fail(TTS_ERR_ARG, "null argument");
    const size_t hdr = 8 * sizeof(int64_t);
    const size_t spin = 3 * size_t(s->n_total) * s->rsize;
    const size_t cells = 2 * size_t(s->ncells_total) * sizeof(double);
    const size_t en = s->n_inst * sizeof(double);
    const size_t oc = s->n_inst * sizeof(int64_t);
    const size_t ring = size_t(s->n_inst) * s->obs_capacity * TTS_NOBS * sizeof(double);
    const size_t need = hdr + spin + cells + en + oc + ring + lattice_state_bytes(s);
    if (!buf) {
        *nbytes = need;
        return TTS_OK;
    }
    if (*nbytes < need) return fail(TTS_ERR_ARG, "state buffer too small");
    if (s->eng) {
        cudaError_t e = engine_sync_to_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine gather");
    }
    TTS_CUDA(cudaStreamSynchronize(s->stream), "get state");
    char *o = static_cast<char *>(buf);
    int64_t h[8] = {0x7474735354415445LL, 1, s->precision, s->n_total, s->n_inst, s->ncells_total, s->obs_capacity, 0};
    TTS_CUDA(cudaMemcpy(&h[7], s->b.step, sizeof(int64_t), cudaMemcpyDeviceToHost), "read step");
    std::memcpy(o, h, hdr);
    o += hdr;
    for (void *arr : {s->b.sx, s->b.sy, s->b.sz}) {
        TTS_CUDA(cudaMemcpy(o, arr, size_t(s->n_total) * s->rsize, cudaMemcpyDeviceToHost), "read spins");
        o += size_t(s->n_total) * s->rsize;
    }
    TTS_CUDA(cudaMemcpy(o, s->b.Te, s->ncells_total * sizeof(double), cudaMemcpyDeviceToHost), "read T_e");
    o += s->ncells_total * sizeof(double);
    TTS_CUDA(cudaMemcpy(o, s->b.Tl, s->ncells_total * sizeof(double), cudaMemcpyDeviceToHost), "read T_l");
    o += s->ncells_total * sizeof(double);
    TTS_CUDA(cudaMemcpy(o, s->b.src_energy, en, cudaMemcpyDeviceToHost), "read energies");
    o += en;
    TTS_CUDA(cudaMemcpy(o, s->b.obs_count, oc, cudaMemcpyDeviceToHost), "read counts");
    o += oc;
    TTS_CUDA(cudaMemcpy(o, s->b.obs_ring, ring, cudaMemcpyDeviceToHost), "read ring");
    o += ring;
    int rc = lattice_state_io(s, o, true);
    if (rc) return rc;
    *nbytes = need;
    return TTS_OK;
}

int tts_set_state(tts_system *s, const void *buf, size_t nbytes)
{
    if (!s || !buf) return fail(TTS_ERR_ARG, "null argument");
    size_t need = 0;
    tts_get_state(s, nullptr, &need);
    if (nbytes != need) return fail(TTS_ERR_ARG, "state size does not match this system");
    const char *o = static_cast<const char *>(buf);
    int64_t h[8];
    std::memcpy(h, o, sizeof h);
    if (h[0] != 0x7474735354415445LL || h[1] != 1 || h[2] != s->precision || h[3] != s->n_total ||
        h[4] != s->n_inst || h[5] != s->ncells_total || h[6] != s->obs_capacity)
        return fail(TTS_ERR_ARG, "state was taken from a different system layout");
    TTS_CUDA(cudaStreamSynchronize(s->stream), "set state");
    o += sizeof h;
    TTS_CUDA(cudaMemcpy(s->b.step, &h[7], sizeof(int64_t), cudaMemcpyHostToDevice), "write step");
    TTS_CUDA(cudaMemset(s->b.open, 0, sizeof(int)), "reset sweep state");
    s->host_step = h[7];
    for (void *arr : {s->b.sx, s->b.sy, s->b.sz}) {
        TTS_CUDA(cudaMemcpy(arr, o, size_t(s->n_total) * s->rsize, cudaMemcpyHostToDevice), "write spins");
        o += size_t(s->n_total) * s->rsize;
    }
    TTS_CUDA(cudaMemcpy(s->b.Te, o, s->ncells_total * sizeof(double), cudaMemcpyHostToDevice), "write T_e");
    o += s->ncells_total * sizeof(double);
    TTS_CUDA(cudaMemcpy(s->b.Tl, o, s->ncells_total * sizeof(double), cudaMemcpyHostToDevice), "write T_l");
    o += s->ncells_total * sizeof(double);
    TTS_CUDA(cudaMemcpy(s->b.src_energy, o, s->n_inst * sizeof(double), cudaMemcpyHostToDevice), "write energies");
    o += s->n_inst * sizeof(double);
    TTS_CUDA(cudaMemcpy(s->b.obs_count, o, s->n_inst * sizeof(int64_t), cudaMemcpyHostToDevice), "write counts");
    o += s->n_inst * sizeof(int64_t);
    TTS_CUDA(cudaMemcpy(s->b.obs_ring, o, size_t(s->n_inst) * s->obs_capacity * TTS_NOBS * sizeof(double),
                        cudaMemcpyHostToDevice), "write ring");
    o += size_t(s->n_inst) * s->obs_capacity * TTS_NOBS * sizeof(double);
    {
        int rc = lattice_state_io(s, const_cast<char *>(o), false);
        if (rc) return rc;
        if ((rc = refresh_sigma(s))) return rc;
    }
    if (s->eng) {
        cudaError_t e = engine_sync_from_general(s->eng, s->b, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "engine scatter");
    }
    return TTS_OK;
}

}  // extern "C"
