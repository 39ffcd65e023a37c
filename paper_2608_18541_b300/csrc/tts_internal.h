// tts_internal.h -- host/device data shared by the runtime and the kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tts.h"

namespace tts {

// SI constants (CODATA 2018).
constexpr double kBoltzmann = 1.380649e-23;        // J/K
constexpr double kBohrMagneton = 9.2740100783e-24; // J/T
constexpr double kGyro = 1.76085963023e11;         // rad s^-1 T^-1
constexpr double kAngstrom = 1e-10;                // m

// ---------------------------------------------------------------------------
// Host-side description of one built instance (canonical atom order).
// ---------------------------------------------------------------------------
struct HostInstance {
    int cells[3] = {1, 1, 1};
    int nbasis = 1;
    int64_t n = 0;
    double box[3] = {0, 0, 0};       // angstrom (lattices)
    std::vector<int> half;           // 3n lattice coordinates in units of a/2
    std::vector<double> pos;         // 3n positions, angstrom
    std::vector<uint8_t> species;    // n
    std::vector<int> colour;         // n
    int ncolours = 1;
    std::vector<int64_t> nbr_begin;  // n + 1
    std::vector<int> nbr;            // neighbour atom ids, ascending per atom
    std::vector<double> nbr_J;       // J_ij, joule
    double frac1 = 0.0;
};

// Build lattice, placement, neighbours and colours of instance `inst`.
// Returns TTS_OK or an error code with *err set.
int build_instance(const tts_system_desc &d, int inst, HostInstance *out, std::string *err);

// Colour-class rule check / greedy colouring (exposed for the resident engine).
void colour_instance(const tts_system_desc &d, HostInstance *hi);

// Message returned by tts_last_error() for the calling thread.
void set_last_error(const std::string &msg);

// ---------------------------------------------------------------------------
// Device-side tables (plain structs copied to device memory).
// ---------------------------------------------------------------------------
constexpr int kMaxColours = 16;

struct DevInstance {
    int64_t slot_begin;                 // first slot of the instance
    int64_t n;                          // atoms
    int64_t colour_begin[kMaxColours + 1]; // slot offsets (relative) of each colour
    int ncolours;
    int cell_begin;                     // first TTM cell (global index)
    int ncells;
    int cells[3];
    int substeps;                       // TTM sub-steps per spin step
    double P0;                          // W m^-3
    double sigma_t, t0;                 // s
    double prof_peak, prof_t1, prof_t2; // step profile: peak T_e (K), end of stage 1, end of stage 2 (s)
    double dx[3];                       // m
    double inv_dx2[3];                  // 1 / dx^2, m^-2
    double cell_volume;                 // m^3
    int obs_block_begin;                // first observable partial block
    int obs_block_count;
};

struct PassRange {
    int64_t slot_begin;                 // global slot
    int64_t count;
    int64_t prefix;                     // exclusive prefix over the pass's ranges
    int inst;
    int hsel;                           // 0: h = dt/2, 1: h = dt
};

struct SpeciesParams {
    double mu;        // J/T
    double inv_mu;    // T/J
    double kappa;     // 2K/mu, tesla
    double alpha;
    double sig_c[2];  // thermal-field scale sqrt(2 alpha k_B / (gamma mu h)), h = dt/2, dt (T in K)
    double gprime;    // gamma / (1 + alpha^2)
    double K;         // J
};

struct TtmParams {
    int active;
    double gamma_e, C_l, G, kappa_e, T0;
    double inv_gamma_e, inv_C_l;
    int source, spatial;
    double sigma_xy, depth_z;   // angstrom
};

}  // namespace tts
