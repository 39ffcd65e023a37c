// tts_noalloc.cu -- a TTM-grid advance that allocates no memory.
//
// Some callers cannot allocate device memory: code whose device memory is all
// owned by another allocator (for example a framework's caching pool that
// holds the whole budget), and latency-critical callers that must not trigger
// cudaMalloc / cudaFree, which can synchronise the whole device.  For them
// tts_ttm_advance_noalloc() advances one two-temperature grid held in the
// caller's own device buffers.  Its only scratch (one double per grid cell
// for the electron-energy increments of a sub-step) lives in the file-scope
// array below, sized for kNoAllocMaxCells cells; every GPU that loads this
// library holds that array (512 KiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "tts_internal.h"

namespace {

constexpr int kNoAllocMaxCells = TTS_NOALLOC_MAX_CELLS;
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device; holds whatever the last call left.  Each
// sub-step writes all of its cells before reading them, so nothing needs
// clearing between calls.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxCells];

std::mutex g_setup_lock;
double *g_scratch_ptr[kNoAllocMaxDevices] = {};

// Same update as the TTM kernel of the general engine (explicit FTCS step of
// gamma_e T_e^2 / 2 with a periodic 7-point Laplacian, e-ph exchange and the
// Gaussian source), for one grid, with the source shape evaluated per cell.
__global__ void ttm_noalloc_kernel(double *__restrict__ Te, double *__restrict__ Tl, double *__restrict__ dE,
                                   int nx, int ny, int nz, double dx0, double dx1, double dx2, double box0,
                                   double box1, double box2, double gamma_e, double C_l, double G, double kappa,
                                   int source, int spatial, double sigma_xy, double depth_z, double P0,
                                   double sigma_t, double t0, double dt, int64_t step, int substeps,
                                   double cell_volume, double *__restrict__ deposited_out)
{
    const int nc = nx * ny * nz;
    const double delta = dt / substeps;
    double deposited = 0.0;
    for (int k = 0; k < substeps; ++k) {
        const double t = double(step) * dt + double(k) * delta;
        double pulse = 0.0;
        if (source != TTS_SOURCE_NONE) {
            const double z = (t - t0) / sigma_t;
            pulse = P0 * exp(-0.5 * z * z);
        }
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
            const double Tc = Te[c];
            double lap = 0.0;
            if (nx > 1)
                lap += (Te[(cz * ny + cy) * nx + (cx + 1) % nx] - 2.0 * Tc + Te[(cz * ny + cy) * nx + (cx + nx - 1) % nx]) /
                       (dx0 * dx0);
            if (ny > 1)
                lap += (Te[(cz * ny + (cy + 1) % ny) * nx + cx] - 2.0 * Tc + Te[(cz * ny + (cy + ny - 1) % ny) * nx + cx]) /
                       (dx1 * dx1);
            if (nz > 1)
                lap += (Te[(((cz + 1) % nz) * ny + cy) * nx + cx] - 2.0 * Tc +
                        Te[(((cz + nz - 1) % nz) * ny + cy) * nx + cx]) / (dx2 * dx2);
            double f = 1.0;
            if (spatial == TTS_SPATIAL_XY_GAUSS) {
                const double rx = (cx + 0.5) * box0 / nx - 0.5 * box0;
                const double ry = (cy + 0.5) * box1 / ny - 0.5 * box1;
                f = exp(-(rx * rx + ry * ry) / (2.0 * sigma_xy * sigma_xy));
            } else if (spatial == TTS_SPATIAL_Z_EXP) {
                f = exp(-((cz + 0.5) * box2 / nz) / depth_z);
            }
            const double src = pulse * f;
            const double x = G * (Tc - Tl[c]);
            dE[c] = delta * (kappa * lap - x + src);
            deposited += delta * src * cell_volume;
            Tl[c] += delta * x / C_l;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const double Ee = 0.5 * gamma_e * Te[c] * Te[c] + dE[c];
            Te[c] = sqrt(2.0 * Ee / gamma_e);
        }
        __syncthreads();
    }
    __shared__ double red[256];
    red[threadIdx.x] = deposited;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && deposited_out) *deposited_out = red[0];
}

int noalloc_fail(int code, const std::string &msg)
{
    tts::set_last_error(msg);   // reported by tts_last_error()
    return code;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device address).
int scratch_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(TTS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(TTS_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_setup_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(TTS_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                                  cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return TTS_OK;
}

}  // namespace

extern "C" {

TTS_API int tts_ttm_advance_noalloc(const tts_ttm_desc *t, const double box_ang[3], double dt, int64_t step,
                                    double *dev_Te, double *dev_Tl, double *dev_deposited, void *stream)
{
    const double P0 = t ? t->P0 : 0.0;
    const double fwhm = t ? t->fwhm : 0.0;
    if (!t || !box_ang || !dev_Te || !dev_Tl) return noalloc_fail(TTS_ERR_ARG, "null argument");
    if (!(dt > 0.0) || step < 0) return noalloc_fail(TTS_ERR_ARG, "dt must be positive and step >= 0");
    int64_t nc = 1;
    for (int k = 0; k < 3; ++k) {
        if (t->cells[k] < 1) return noalloc_fail(TTS_ERR_ARG, "TTM cell counts must be >= 1");
        if (!(box_ang[k] > 0.0)) return noalloc_fail(TTS_ERR_ARG, "box edges must be positive");
        // checked before multiplying, so that the product cannot overflow
        if (t->cells[k] > kNoAllocMaxCells / nc)
            return noalloc_fail(TTS_ERR_ARG, "grid has more than " + std::to_string(kNoAllocMaxCells) +
                                                 " cells; this entry point handles at most " +
                                                 std::to_string(kNoAllocMaxCells));
        nc *= t->cells[k];
    }
    if (nc > kNoAllocMaxCells)
        return noalloc_fail(TTS_ERR_ARG, "grid has " + std::to_string(nc) + " cells; this entry point handles at most " +
                                             std::to_string(kNoAllocMaxCells));
    if (!(t->gamma_e > 0.0) || !(t->C_l > 0.0) || !(t->G >= 0.0) || !(t->kappa_e >= 0.0) || !(t->T0 > 0.0))
        return noalloc_fail(TTS_ERR_ARG, "TTM coefficients out of range");
    if (t->source < 0 || t->source > 2 || t->spatial < 0 || t->spatial > 2) return noalloc_fail(TTS_ERR_ARG, "bad TTM mode");
    if (t->source != TTS_SOURCE_NONE && !(fwhm > 0.0)) return noalloc_fail(TTS_ERR_ARG, "pulse FWHM must be positive");
    if (t->spatial == TTS_SPATIAL_XY_GAUSS && !(t->sigma_xy > 0.0))
        return noalloc_fail(TTS_ERR_ARG, "the Gaussian spot needs sigma_xy > 0");
    if (t->spatial == TTS_SPATIAL_Z_EXP && !(t->depth_z > 0.0))
        return noalloc_fail(TTS_ERR_ARG, "the exponential profile needs depth_z > 0");
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // geometry and sub-steps as in tts_set_ttm_grid: dt/m <= 0.4 C_e(T0) dx_min^2 / (kappa_e d)
    double dx[3], vol = 1.0, dxmin = 0.0;
    int resolved = 0;
    for (int k = 0; k < 3; ++k) {
        dx[k] = box_ang[k] * tts::kAngstrom / t->cells[k];
        vol *= dx[k];
        if (t->cells[k] > 1) {
            dxmin = resolved ? (dx[k] < dxmin ? dx[k] : dxmin) : dx[k];
            ++resolved;
        }
    }
    int substeps = 1;
    if (resolved > 0 && t->kappa_e > 0.0) {
        const double m = std::ceil(dt / (0.4 * t->gamma_e * t->T0 * dxmin * dxmin / (t->kappa_e * resolved)));
        substeps = m < 1.0 ? 1 : static_cast<int>(m);
    }
    const double sigma_t = t->source != TTS_SOURCE_NONE ? fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0))) : 1.0;
    const double t0 = t->t0 >= 0.0 ? t->t0 : 3.0 * sigma_t;
    ttm_noalloc_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        dev_Te, dev_Tl, scratch, t->cells[0], t->cells[1], t->cells[2], dx[0], dx[1], dx[2], box_ang[0], box_ang[1],
        box_ang[2], t->gamma_e, t->C_l, t->G, t->kappa_e, t->source, t->spatial, t->sigma_xy, t->depth_z, P0, sigma_t,
        t0, dt, step, substeps, vol, dev_deposited);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(TTS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return TTS_OK;
}

}  // extern "C"
