// Internal interface between the batch driver (api.cu) and the serving loop
// (server.cu): one Newton round over an active set of cells, per-cell trial
// state, the Newton test, and the final commit of finished cells.
#pragma once

#include <stdint.h>

#include "../../include/fftg.h"

namespace fftg_detail {

// Scalars of one cell after one Newton round.
struct RoundOut {
    int cg_it = 0;        // CG iterations of the round's solve
    int cg_done = 0;      // how the solve ended (CG_* status)
    double de2 = 0.0;     // ||d eps||^2
    double gs2 = 0.0;     // ||G sigma||^2
    double sig2 = 0.0;    // ||sigma||^2
    double relres = 0.0;  // final ||r|| / ||r0||
};

// One Newton iteration (constitutive, residual, CG, eps* += d eps) for
// every cell with run[cell] != 0, all in the same launches.
int newton_round(fftg_handle* h, const int* run, double tol_inner, RoundOut* out);

// Set a cell's trial macroscopic strain; with copy_eps, start its working
// fluctuation from the committed one (the start of an increment).
int set_trial_strain(fftg_handle* h, int cell, const double Et[6], bool copy_eps);

// Newton test of one cell after a round: 0 = keep iterating, 1 = converged,
// negative = FFTG_E* failure. Records the round in the cell's stats.
int newton_decide(fftg_handle* h, int cell, const RoundOut& ro, double normE, double tol_newton, int* it);

// Final constitutive call, homogenised stress (sigma_out[6*cell..]) and
// commit of every cell with fin[cell] != 0.
int finish_cells(fftg_handle* h, const int* fin, double* sigma_out);

// Replace a cell's microstructure (phase != null) and committed state
// (state = E[6], eps*[6V], eps_p[6V], epbar[V]; null = zero state).
int upload_cell(fftg_handle* h, int cell, const uint8_t* phase, const double* state);
int download_cell(fftg_handle* h, int cell, double* state);

void reset_stats(fftg_handle* h, int cell);
void set_status(fftg_handle* h, int cell, int status);

int cells(const fftg_handle* h);
int grid_n(const fftg_handle* h);
bool is_mixed(const fftg_handle* h);
const fftg_options& options(const fftg_handle* h);
const double* committed_E(const fftg_handle* h, int cell);
long long voxels(const fftg_handle* h);

}  // namespace fftg_detail
