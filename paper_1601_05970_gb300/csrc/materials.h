// Host-side checks and packing of the phase records (fftg_phase) into the
// device material table of the constitutive kernel.
#pragma once

#include <cmath>

#include "../../include/fftg.h"
#include "common.cuh"

namespace fftg {

static_assert(MODEL_J2 == FFTG_MODEL_J2 && MODEL_NLELASTIC == FFTG_MODEL_NLELASTIC &&
                  MODEL_VISCO == FFTG_MODEL_VISCO,
              "model ids");

inline bool pos_finite(double v) { return v > 0.0 && std::isfinite(v); }

// Parameters of each model as fftg.h states them; rate-dependent phases
// only where the caller has a time step.
inline bool phase_valid(const fftg_phase& m, bool rate_ok) {
    switch (m.model) {
        case FFTG_MODEL_J2:
            return pos_finite(m.K) && pos_finite(m.G) && m.sigma_y > 0.0 && m.H >= 0.0 &&
                   std::isfinite(m.H) && pos_finite(m.n);
        case FFTG_MODEL_NLELASTIC:
            return pos_finite(m.K) && pos_finite(m.sigma_y) && pos_finite(m.eps0) && pos_finite(m.n);
        case FFTG_MODEL_VISCO:
            return rate_ok && pos_finite(m.K) && pos_finite(m.G) && pos_finite(m.sigma_y) &&
                   pos_finite(m.eps0) && pos_finite(m.t0) && pos_finite(m.n);
        default:
            return false;
    }
}

inline void pack_phase(const fftg_phase& m, double* row) {
    row[0] = m.K;
    row[1] = m.G;
    row[2] = m.sigma_y;
    row[3] = m.H;
    row[4] = m.n;
    row[5] = m.eps0;
    row[6] = m.t0;
    row[7] = (double)m.model;
}

}  // namespace fftg
