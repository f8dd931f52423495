// Device-side control of one load increment of a batch of cells, so that
// the whole increment (Newton loop, CG loops, commit) runs as one CUDA
// graph launch with no host round trip: the Newton test of Algorithm 1
// (||d eps|| / ||E||_field <= eta_NW, at least one iteration, the caps and
// the failure cases of the host driver) is taken per cell by a one-block
// kernel that also sets the condition of the graph's Newton loop.
#pragma once

#include "../../include/fftg.h"
#include "common.cuh"

namespace fftg {

// Per-cell state of the increment run on the device.
struct IncDev {
    double normE;      // sqrt(V) ||E_trial||_F
    double sigma[6];   // homogenised stress of the converged increment
    int newton;        // Newton iterations taken
    int cg;            // CG iterations summed over them
    int state;         // INC_*
    int status;        // FFTG_OK or the failure code
};

enum : int { INC_IDLE = 0, INC_NEWTON = 1, INC_DONE = 2, INC_FAILED = 3 };

struct IncArgs {
    int B;                 // cells
    long long V;           // voxels per cell
    const int* run;        // [B] cells taking part in this increment
    const double* dE;      // [B][6] increments (device copy of the host's)
    double* Ecom;          // [B][6] committed macroscopic strain
    double* Etrial;        // [B][6] trial macroscopic strain (the Edev of the kernels)
    int* active;           // [B] cells iterating Newton
    int* fin;              // [B] cells to commit
    IncDev* inc;           // [B]
    CGState* cg;           // [B]
    CGState cg_template;   // tolerance, caps and stagnation window of a solve
    const NewtonDev* nd;   // [B] de2 after the Newton update; sums after the commit update
    double tol_newton;
    int max_newton;
    int fixed_newton;
    unsigned int* newton_guard;  // Newton loop passes of the increment
    unsigned int* cg_guard;      // CG loop passes of the solve (k_cg_continue's counter)
    unsigned int newton_cap;
};

// Start of the increment: trial strain E + dE, ||E||_field, counters; the
// Newton loop's condition starts true.
__global__ void k_inc_begin(cudaGraphConditionalHandle newton_cond, IncArgs a) {
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        IncDev& s = a.inc[b];
        s.newton = 0;
        s.cg = 0;
        s.status = FFTG_OK;
        const bool on = a.run[b] != 0;
        s.state = on ? INC_NEWTON : INC_IDLE;
        a.active[b] = on ? 1 : 0;
        a.fin[b] = 0;
        double e[6];
        for (int c = 0; c < 6; ++c) {
            e[c] = a.Ecom[6 * b + c] + (on ? a.dE[6 * b + c] : 0.0);
            a.Etrial[6 * b + c] = e[c];
        }
        s.normE = sqrt((double)a.V) * sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2] +
                                           2.0 * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]));
    }
    if (threadIdx.x == 0) {
        *a.newton_guard = 0u;
        cudaGraphSetConditional(newton_cond, 1u);
    }
}

// Start of a Newton iteration: fresh CG states for the active cells (the
// others are marked converged, so their CG kernels return at entry); the
// CG loop's condition starts true.
__global__ void k_inc_cg_reset(cudaGraphConditionalHandle cg_cond, IncArgs a) {
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        CGState c = a.cg_template;
        c.done = a.active[b] ? CG_RUNNING : CG_CONVERGED;
        a.cg[b] = c;
    }
    if (threadIdx.x == 0) {
        *a.cg_guard = 0u;
        cudaGraphSetConditional(cg_cond, 1u);
    }
}

// After the Newton update: the test of each active cell, and the condition
// of the Newton loop (any cell still active; at most newton_cap passes).
__global__ void k_inc_decide(cudaGraphConditionalHandle cond, IncArgs a) {
    int any = 0;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        if (!a.active[b]) continue;
        IncDev& s = a.inc[b];
        const CGState& c = a.cg[b];
        s.newton += 1;
        s.cg += c.it;
        const double nde = sqrt(a.nd[b].de2);
        const double rel = s.normE > 0.0 ? nde / s.normE : (nde == 0.0 ? 0.0 : INFINITY);
        int verdict = 0;  // 0 iterate, 1 converged, < 0 failed
        if (c.done == CG_BREAKDOWN || !isfinite(rel))
            verdict = FFTG_ENAN;
        else if (a.fixed_newton > 0)
            verdict = s.newton >= a.fixed_newton ? 1 : 0;
        else if (rel <= a.tol_newton || nde == 0.0)
            verdict = 1;
        else if (s.newton >= a.max_newton)
            verdict = FFTG_ENOCONV_NEWTON;
        if (verdict == 1) {
            s.state = INC_DONE;
            a.active[b] = 0;
            a.fin[b] = 1;
        } else if (verdict < 0) {
            s.state = INC_FAILED;
            s.status = verdict;
            a.active[b] = 0;
        } else {
            any = 1;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        const unsigned int n = ++*a.newton_guard;
        cudaGraphSetConditional(cond, (any && n < a.newton_cap) ? 1u : 0u);
    }
}

// After the commit's stress update: the homogenised stress of the
// finished cells and their committed macroscopic strain.
__global__ void k_inc_end(IncArgs a) {
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        if (!a.fin[b]) continue;
        for (int c = 0; c < 6; ++c) {
            a.inc[b].sigma[c] = a.nd[b].sum[c] / (double)a.V;
            a.Ecom[6 * b + c] = a.Etrial[6 * b + c];
        }
    }
}

// Commit of the finished cells: trial state -> committed state (eps*,
// plastic strain, accumulated plastic strain), one grid over the cells.
struct CommitArgs {
    const int* fin;
    double* eps_star;
    const double* eps_work;
    double* eps_p;
    const double* eps_p_tr;
    double* epbar;
    const double* epbar_tr;
    long long cs;          // component stride; a cell's fields are [6][cs], its epbar [cs]
};

__global__ void k_inc_commit(CommitArgs a) {
    const int b = blockIdx.y;
    if (!a.fin[b]) return;
    const long long n6 = 6 * a.cs;
    const long long f = (long long)b * n6, e = (long long)b * a.cs;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n6;
         i += (long long)gridDim.x * blockDim.x) {
        a.eps_star[f + i] = a.eps_work[f + i];
        a.eps_p[f + i] = a.eps_p_tr[f + i];
        if (i < a.cs) a.epbar[e + i] = a.epbar_tr[e + i];
    }
}

}  // namespace fftg
