// Pointwise kernels of the Newton-CG path: the J2 return mapping with its
// consistent tangent (Section 4.2), the CG vector updates (Hestenes-Stiefel)
// with their reductions, the Newton update eps* += d eps (Algorithm 1), and
// the reductions of the macroscopic tangent.
#pragma once

#include <cfloat>

#include "common.cuh"
#include "passes.cuh"

namespace fftg {

// Maximum grid of the grid-stride pointwise kernels (fixed per V, so the
// reduction order never depends on timing).
constexpr int kMaxPointwiseBlocks = 4096;

inline int pointwise_blocks(long long V) {
    long long b = (V + kThreads - 1) / kThreads;
    return (int)(b < kMaxPointwiseBlocks ? b : kMaxPointwiseBlocks);
}

// Grid of the vectorised CG update: one thread per 16-byte vector up to a
// fixed cap (depends only on the grid size).
inline int vector_blocks(long long cs, int elem_bytes) {
    const long long nv = cs / (16 / elem_bytes);
    long long b = (nv + kThreads - 1) / kThreads;
    return (int)(b < 2432 ? b : 2432);
}

struct ConstArgs {
    long long V;
    long long cs;            // component stride of the fields (>= V)
    double E[6];
    const double* eps;       // [6][V] fluctuation eps*
    const double* eps_p;     // [6][V] committed plastic strain
    const double* epbar;     // [V] committed accumulated plastic strain
    const uint8_t* phase;    // [V]
    const double* mats;      // [nphase][kMatStride]: K, G, sigma_0, H, n, eps_0, t_0, model
    double* sigma;           // [6][V] out (may be null)
    double* eps_p_new;       // [6][V] out (may be null)
    double* epbar_new;       // [V] out (may be null)
    void* tangent;           // [7][V] out in TT (may be null)
    double* partials;        // [nblocks][7]
    NewtonDev* nd;           // sig2 and sum of sigma
    CGState* cg;             // if set: cg->floor2 from ||sigma||
    double tie;              // plastic iff Phi_trial > tie * sigma_y
    double dt;               // time step of the increment (visco-plastic phases)
    int skip_sums;           // 1: nd->sum (the sums of sigma) is left at 0; only the
                             // commit's call, which writes the history, needs it
    int elastic_only;        // 1: J2 and visco-plastic phases skip the return
                             // (sigma = C_e : (eps - eps_p), the stress of a
                             // committed state); non-linear elastic phases
                             // are evaluated as usual
    // Batches of cells: cell = blockIdx.y; per-cell offsets below (0 for a
    // single cell). Edev [cells][6] replaces E when set; active[cell] == 0
    // skips the cell.
    const double* Edev;
    const int* active;
    long long cell_fields;   // stride between cells of the [6][cs] fields
    long long cell_scalar;   // stride of epbar / phase between cells
    long long cell_tangent;  // stride of the tangent between cells
};

// Root dgamma of the scalar return equation of Section 4.2,
//   seq - 3 G dgamma - sigma_0 - H (epbar_t + dgamma)^n = 0,
// for a trial state with Phi_tr = phi > 0. The left side is positive at 0
// and non-positive at phi / (3G) (the hardening term only grows), so the
// root is bracketed there; Newton steps that leave the current bracket are
// replaced by bisection. Stops when the step or the bracket is at the last
// few bits, after at most 100 iterations.
__device__ __forceinline__ double power_law_return(double seq, double eb, double G, double sy,
                                                   double Hh, double n, double phi) {
    double lo = 0.0, hi = phi / (3.0 * G);
    double x = 0.5 * hi;
    for (int k = 0; k < 100; ++k) {
        const double y = eb + x;
        const double yn = pow(y, n);
        const double f = seq - 3.0 * G * x - sy - Hh * yn;
        if (f > 0.0) lo = x; else hi = x;
        const double df = -3.0 * G - (y > 0.0 ? n * Hh * yn / y : (double)INFINITY);
        double xn = x - f / df;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const bool done = fabs(xn - x) <= 4.0 * DBL_EPSILON * x || hi - lo <= 4.0 * DBL_EPSILON * hi;
        x = xn;
        if (done) break;
    }
    return x;
}

// Material update at every voxel by its phase's model: non-linear
// elasticity (Section 4.1), or for J2 (Section 4.2, hardening
// sigma_0 + H epbar^n) and visco-plasticity (Section 4.3) the elastic
// predictor / plastic corrector:
// trial sigma = C_e : (eps - eps_p^t); Phi = sigma_eq - (sigma_y + H (epbar^t)^n);
// if Phi > tie*sigma_y: dgamma from the scalar return equation (closed form
// Phi / (3G + H) for n = 1), N = 3/2 s / sigma_eq, eps_p += dgamma N,
// epbar += dgamma, sigma -= 2G dgamma N, and the tangent
// C = C_e - 6G^2 dgamma/sigma_eq I_d + 4G^2 (dgamma/sigma_eq - 1/(3G + h')) N(x)N,
// h' = n H (epbar^t + dgamma)^(n-1), stored as K', 2G_eff, w = sqrt(|b|) N
// with b the N(x)N coefficient and K' = K for b <= 0 (always for n <= 1),
// K' = -K for b > 0.
// Two blocks per SM (at most 128 registers): unbounded, the kernel takes
// about 155 registers and runs one block per SM, 5 % slower at 243^3.
template <typename TT>
__global__ void __launch_bounds__(kThreads, 2) k_constitutive(ConstArgs a) {
    const int cell = blockIdx.y;
    if (a.active && !a.active[cell]) return;
    const long long V = a.V, cs = a.cs;
    const long long of = cell * a.cell_fields, osc = cell * a.cell_scalar;
    double E[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) E[c] = a.Edev ? a.Edev[6 * cell + c] : a.E[c];
    const double* eps = a.eps + of;
    const double* eps_p = a.eps_p + of;
    const double* epbar = a.epbar + osc;
    const uint8_t* phase = a.phase + osc;
    double* sigma = a.sigma ? a.sigma + of : nullptr;
    double* eps_p_new = a.eps_p_new ? a.eps_p_new + of : nullptr;
    double* epbar_new = a.epbar_new ? a.epbar_new + osc : nullptr;
    NewtonDev* nd = a.nd + cell;
    double* partials = a.partials + (size_t)cell * gridDim.x * 7;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    TT* tg = a.tangent ? (TT*)a.tangent + cell * a.cell_tangent : nullptr;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        const int ph = phase[v];
        const double* mp = a.mats + kMatStride * ph;
        const double K = mp[0], G = mp[1], sy = mp[2], nh = mp[4];
        const int model = (int)mp[7];
        // elastic trial strain; the non-linear elastic model uses the total
        // strain (it has no plastic strain; eps_p passes through unchanged)
        const bool nle = model == MODEL_NLELASTIC;
        double e[6], ep[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ep[c] = eps_p[c * cs + v];
            e[c] = E[c] + eps[c * cs + v] - (nle ? 0.0 : ep[c]);
        }
        const double eb = epbar[v];
        const double tr = e[0] + e[1] + e[2];
        const double m = tr * (1.0 / 3.0);
        double sig[6];
        TT g2t;  // 2G_eff of the tangent, in the tangent's precision
        TT w[6] = {TT(0), TT(0), TT(0), TT(0), TT(0), TT(0)};  // in the tangent's precision
        double dg = 0.0;
        bool kneg = false;  // N(x)N coefficient of the tangent positive
        if (nle) {
            // Section 4.1: sigma_d = sigma_0 (eps_eq/eps_0)^n N, N = 2/3 d/eps_eq,
            // d = dev(eps), eps_eq = sqrt(2/3 d:d); tangent
            // c ((n - 1) N(x)N + 2/3 I_d), c = sigma_0/eps_eq (eps_eq/eps_0)^n,
            // whose limit at eps_eq = 0 is taken as sigma_0/eps_0 for n = 1, else 0
            const double d[6] = {e[0] - m, e[1] - m, e[2] - m, e[3], e[4], e[5]};
            const double eeq = sqrt((2.0 / 3.0) * frob<double>(d, d));
            const double e0r = mp[5];
            const double c = eeq > 0.0 ? sy / eeq * pow(eeq / e0r, nh) : (nh == 1.0 ? sy / e0r : 0.0);
            const double g2 = (2.0 / 3.0) * c;
            g2t = (TT)g2;
#pragma unroll
            for (int k = 0; k < 6; ++k) sig[k] = g2 * d[k];
            const double b = c * (nh - 1.0);
            kneg = b > 0.0;
            const double sbN = eeq > 0.0 ? sqrt(fabs(b)) * (2.0 / 3.0) / eeq : 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) w[k] = (TT)(sbN * d[k]);
        } else {
            // J2 (Section 4.2) or visco-plasticity (Section 4.3), elastic
            // trial state. The visco-plastic backward-Euler equation
            // seq - 3G dgamma = sigma_0 (dgamma / (gamma_0 dt))^n has the
            // form of the J2 return with no yield stress, no history in the
            // rate term and H = sigma_0 (gamma_0 dt)^(-n), gamma_0 = eps_0/t_0.
            const bool visco = model == MODEL_VISCO;
            const double g2e = 2.0 * G;
            double s[6];
            s[0] = g2e * (e[0] - m);
            s[1] = g2e * (e[1] - m);
            s[2] = g2e * (e[2] - m);
            s[3] = g2e * e[3];
            s[4] = g2e * e[4];
            s[5] = g2e * e[5];
            const double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] +
                              2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
            const double seq = sqrt(1.5 * ss);
            const double sy_h = visco ? 0.0 : sy;
            const double Hh = visco ? sy * pow(mp[5] / mp[6] * a.dt, -nh) : mp[3];
            const double eb_h = visco ? 0.0 : eb;
            const bool linear = nh == 1.0;
            const double phi = seq - (sy_h + Hh * (linear ? eb_h : pow(eb_h, nh)));
            g2t = (TT)g2e;
            if (!a.elastic_only && phi > a.tie * sy) {
                double inv_seq, inv_h3;
                if (linear) {
                    // one division gives both 1/sigma_eq and 1/(3G + H)
                    const double h3 = 3.0 * G + Hh;
                    const double rr = 1.0 / (seq * h3);
                    inv_seq = rr * h3;
                    inv_h3 = rr * seq;
                    dg = phi * inv_h3;
                } else {
                    dg = power_law_return(seq, eb_h, G, sy_h, Hh, nh, phi);
                    const double y = eb_h + dg;  // > 0: dg > 0 on a plastic step
                    inv_seq = 1.0 / seq;
                    inv_h3 = 1.0 / (3.0 * G + nh * Hh * pow(y, nh - 1.0));
                }
                const double f = 1.5 * inv_seq;
                const double gdg = g2e * dg;
                const double dgs = dg * inv_seq;
                const double bd = dgs - inv_h3;  // b = 4 G^2 bd
                if (bd > 0.0) kneg = true;
                if constexpr (sizeof(TT) == 4) {
                    // FP32 tangent: N = f s is not formed (sigma = (1 - 2G dgamma f) s,
                    // eps_p += dgamma f s), and the tangent's coefficients and
                    // w = sqrt(|b|) N, stored in FP32, are formed in FP32; the
                    // kernel is bound by FP64 arithmetic
                    const double c1 = 1.0 - gdg * f, c2 = dg * f;
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        sig[c] = c1 * s[c];
                        ep[c] += c2 * s[c];
                    }
                    const float Gf = (float)G, dgsf = (float)dgs;
                    g2t = 2.0f * Gf - 6.0f * Gf * Gf * dgsf;
                    const float sf = sqrtf(4.0f * Gf * Gf * fabsf((float)bd)) * (float)f;
#pragma unroll
                    for (int c = 0; c < 6; ++c) w[c] = sf * (float)s[c];
                } else {
                    g2t = (TT)(g2e - 6.0 * G * G * dgs);
                    const double b = 4.0 * G * G * bd;
                    double Nn[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Nn[c] = f * s[c];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        sig[c] = s[c] - gdg * Nn[c];
                        ep[c] += dg * Nn[c];
                    }
                    const double sb = sqrt(fabs(b));
#pragma unroll
                    for (int c = 0; c < 6; ++c) w[c] = (TT)(sb * Nn[c]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) sig[c] = s[c];
            }
        }
        const double kt = K * tr;
        sig[0] += kt;
        sig[1] += kt;
        sig[2] += kt;
        if (sigma) {
#pragma unroll
            for (int c = 0; c < 6; ++c) sigma[c * cs + v] = sig[c];
        }
        if (eps_p_new) {
#pragma unroll
            for (int c = 0; c < 6; ++c) eps_p_new[c * cs + v] = ep[c];
        }
        if (epbar_new) epbar_new[v] = eb + dg;
        if (tg) {
            tg[v] = (TT)(kneg ? -K : K);
            tg[cs + v] = g2t;
            tg[2 * cs + v] = w[0];
            tg[3 * cs + v] = w[1];
            tg[4 * cs + v] = w[3];
            tg[5 * cs + v] = w[4];
            tg[6 * cs + v] = w[5];
        }
        acc[0] += frob<double>(sig, sig);
        if (!a.skip_sums) {
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[1 + c] += sig[c];
        }
    }
    double part[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) part[j] = block_sum(acc[j]);
    if (!publish_partials<7>(part, partials, blockIdx.x, gridDim.x, &nd->ticket)) return;
    double tot[7];
    reduce_partials<7>(partials, gridDim.x, &nd->ticket, tot);
    if (threadIdx.x == 0) {
        nd->sig2 = tot[0];
        for (int c = 0; c < 6; ++c) nd->sum[c] = tot[1 + c];
        if (a.cg) a.cg[cell].floor2 = kRoundoffRel * kRoundoffRel * tot[0];
    }
}

struct VecArgs {
    long long V;
    long long cs;      // component stride (a multiple of 32, >= V + 4)
    void* x;
    void* r;
    const void* p;
    const void* q;
    double* eps;       // newton update: eps* (FP64)
    CGState* cg;
    NewtonDev* nd;
    double* partials;  // [nf][nblocks][NV]
    long long fstride;
    const void* tangent;
    double* out;       // tangent averages
    const int* active; // per cell (newton update): 0 = skip
    long long cell_fields;  // stride between cells of eps (newton update)
    long long cell_tangent; // stride between cells of the tangent (bounds)
    int nw;                 // CG states written per cell (bounds)
};

// r -= alpha q; rr = <r, r>; then beta, stopping test. The matching step
// x += alpha p is deferred: the next iteration's P1 adds it while it reads
// p anyway, and k_cg_finish adds the last one (CGState::pend), so x costs
// no extra pass over memory.
// 16-byte vectors over the padded components; lanes in the padding are
// updated too (harmless) but left out of <r, r>.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_update(VecArgs a) {
    const int f = blockIdx.z;
    CGState* cg = a.cg + f;
    if (cg->done) return;
    constexpr int VW = 16 / (int)sizeof(T);
    using VT = typename Vec16<T>::type;
    const long long V = a.V, cs = a.cs;
    const long long nv = cs / VW;
    const T alpha = (T)cg->alpha;
    VT* r = (VT*)((T*)a.r + f * a.fstride);
    const VT* q = (const VT*)((const T*)a.q + f * a.fstride);
    T acc = T(0);
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < nv;
         j += (long long)gridDim.x * kThreads) {
        T rv[6][VW];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            VT rr = r[c * nv + j];
            const VT qv = q[c * nv + j];
            T* re = reinterpret_cast<T*>(&rr);
            const T* qe = reinterpret_cast<const T*>(&qv);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                re[e] -= alpha * qe[e];
                rv[c][e] = re[e];
            }
            r[c * nv + j] = rr;
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            if (j * VW + e < V) {
                const T re6[6] = {rv[0][e], rv[1][e], rv[2][e], rv[3][e], rv[4][e], rv[5][e]};
                acc += frob<T>(re6, re6);
            }
        }
    }
    double part[1] = {block_sum((double)acc)};
    double* partials = a.partials + (size_t)f * gridDim.x;
    if (!publish_partials<1>(part, partials, blockIdx.x, gridDim.x, &cg->ticket)) return;
    double tot[1];
    reduce_partials<1>(partials, gridDim.x, &cg->ticket, tot);
    if (threadIdx.x != 0) return;
    cg_after_update(cg, tot[0]);
}

// After the last CG iteration: x += alpha p where the last update left the
// step pending.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_finish(VecArgs a) {
    const int f = blockIdx.z;
    const CGState* cg = a.cg + f;
    if (!cg->pend) return;
    constexpr int VW = 16 / (int)sizeof(T);
    using VT = typename Vec16<T>::type;
    const long long nv = 6 * a.cs / VW;
    const T alpha = (T)cg->alpha;
    VT* x = (VT*)((T*)a.x + f * a.fstride);
    const VT* p = (const VT*)((const T*)a.p + f * a.fstride);
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < nv;
         j += (long long)gridDim.x * kThreads) {
        VT xv = x[j];
        const VT pv = p[j];
        T* xe = reinterpret_cast<T*>(&xv);
        const T* pe = reinterpret_cast<const T*>(&pv);
#pragma unroll
        for (int e = 0; e < VW; ++e) xe[e] += alpha * pe[e];
        x[j] = xv;
    }
}

// eps* += x (Algorithm 1, iterative update); nd->de2 = ||x||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_newton_update(VecArgs a) {
    const int cell = blockIdx.y;
    if (a.active && !a.active[cell]) return;
    const long long V = a.V, cs = a.cs;
    const T* x = (const T*)a.x + cell * a.fstride;
    double* eps = a.eps + cell * a.cell_fields;
    NewtonDev* nd = a.nd + cell;
    double* partials = a.partials + (size_t)cell * gridDim.x;
    double acc = 0.0;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        double d[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            d[c] = (double)x[c * cs + v];
            eps[c * cs + v] += d[c];
        }
        acc += frob<double>(d, d);
    }
    double part[1] = {block_sum(acc)};
    if (!publish_partials<1>(part, partials, blockIdx.x, gridDim.x, &nd->ticket)) return;
    double tot[1];
    reduce_partials<1>(partials, gridDim.x, &nd->ticket, tot);
    if (threadIdx.x == 0) nd->de2 = tot[0];
}

// s = C : p at voxel v with the compact tangent in the tangent's precision
template <typename T>
__device__ __forceinline__ void tangent_apply_v(const T* __restrict__ tg, long long v, long long cs,
                                                const T (&p)[6], T (&s)[6]) {
    apply_tangent7<T>(tg[v], tg[cs + v], tg[2 * cs + v], tg[3 * cs + v], tg[4 * cs + v],
                      tg[5 * cs + v], tg[6 * cs + v], p, s);
}

// Roundoff floors of the six tangent right-hand sides: ||C : E_j||^2.
// Products in the tangent's precision, per-thread sums in T, block sums and
// the total in FP64 (only the order of magnitude matters for a floor).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tangent_floor(VecArgs a) {
    const long long V = a.V;
    const T* tg = (const T*)a.tangent;
    T acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            T e[6] = {0, 0, 0, 0, 0, 0}, s[6];
            e[j] = T(1);
            tangent_apply_v<T>(tg, v, a.cs, e, s);
            acc[j] += frob<T>(s, s);
        }
    }
    double part[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) part[j] = block_sum((double)acc[j]);
    if (!publish_partials<6>(part, a.partials, blockIdx.x, gridDim.x, &a.nd->ticket)) return;
    double tot[6];
    reduce_partials<6>(a.partials, gridDim.x, &a.nd->ticket, tot);
    if (threadIdx.x == 0)
        for (int j = 0; j < 6; ++j) a.cg[j].floor2 = kRoundoffRel * kRoundoffRel * tot[j];
}

// out[i*6 + j] = sum over voxels of (C : (E_j + x_j))_i. C : (E_j + x_j) is
// formed in the precision of the tangent and of x (FP32 in the mixed path,
// where both are FP32); each thread sums its few voxels in that precision
// and the block and grid sums are FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tangent_average(VecArgs a) {
    const long long V = a.V;
    const T* tg = (const T*)a.tangent;
    const T* x = (const T*)a.x;
    T acc[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) acc[k] = T(0);
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            T e[6], s[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) e[c] = x[j * a.fstride + c * a.cs + v] + (c == j ? T(1) : T(0));
            tangent_apply_v<T>(tg, v, a.cs, e, s);
#pragma unroll
            for (int i = 0; i < 6; ++i) acc[i * 6 + j] += s[i];
        }
    }
    double part[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) part[k] = block_sum((double)acc[k]);
    if (!publish_partials<36>(part, a.partials, blockIdx.x, gridDim.x, &a.nd->ticket)) return;
    double tot[36];
    reduce_partials<36>(a.partials, gridDim.x, &a.nd->ticket, tot);
    if (threadIdx.x == 0)
        for (int k = 0; k < 36; ++k) a.out[k] = tot[k];
}

// The basic scheme (Section 3.2, Moulinec-Suquet) solves the linear system
// by Richardson's iteration with the reference medium
// C_ref = (lambda_min + lambda_max)/2 I_s, lambda the extreme eigenvalues
// of the local tangents over the grid; with Gamma_ref = G / c for
// C_ref = c I_s (Appendix A), this is Richardson's iteration on G C with
// the step omega = 2 / (lambda_min + lambda_max). On symmetric tensors with
// the Frobenius product the compact tangent |K'| I(x)I + 2G_eff I_d + b N(x)N
// has the eigenvalues 3|K'| (spherical), 2G_eff (deviatoric, orthogonal to
// w) and 2G_eff - sign(K') |w|^2 (along w). The last block writes omega into
// the nw CG states of the cell; it runs after the right-hand side pass (which
// resets the states) and before the iteration.
__device__ __forceinline__ void block_minmax(double& lo, double& hi) {
    __shared__ double slo[kThreads / 32], shi[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        slo[wid] = lo;
        shi[wid] = hi;
    }
    __syncthreads();
    lo = slo[0];
    hi = shi[0];
    for (int k = 1; k < kThreads / 32; ++k) {
        lo = fmin(lo, slo[k]);
        hi = fmax(hi, shi[k]);
    }
}

template <typename TT>
__global__ void __launch_bounds__(kThreads) k_tangent_bounds(VecArgs a) {
    const int cell = blockIdx.y;
    if (a.active && !a.active[cell]) return;
    const long long V = a.V, cs = a.cs;
    const TT* tg = (const TT*)a.tangent + cell * a.cell_tangent;
    double lo = INFINITY, hi = -INFINITY;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        const double Kp = tg[v], g2 = tg[cs + v];
        const double w0 = tg[2 * cs + v], w1 = tg[3 * cs + v], w3 = tg[4 * cs + v],
                     w4 = tg[5 * cs + v], w5 = tg[6 * cs + v];
        const double w2 = -(w0 + w1);
        const double ww = w0 * w0 + w1 * w1 + w2 * w2 + 2.0 * (w3 * w3 + w4 * w4 + w5 * w5);
        const double l1 = 3.0 * fabs(Kp), l3 = Kp < 0.0 ? g2 + ww : g2 - ww;
        lo = fmin(lo, fmin(l1, fmin(g2, l3)));
        hi = fmax(hi, fmax(l1, fmax(g2, l3)));
    }
    block_minmax(lo, hi);
    double* partials = a.partials + (size_t)cell * gridDim.x * 2;
    NewtonDev* nd = a.nd + cell;
    const double part[2] = {lo, hi};
    if (!publish_partials<2>(part, partials, blockIdx.x, gridDim.x, &nd->ticket)) return;
    __threadfence();
    lo = INFINITY;
    hi = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        lo = fmin(lo, __ldcg(partials + 2 * (size_t)b));
        hi = fmax(hi, __ldcg(partials + 2 * (size_t)b + 1));
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        nd->ticket = 0u;
        // the scheme needs positive definite tangents: otherwise the solve
        // stops as a breakdown
        const bool ok = lo > 0.0 && isfinite(hi);
        for (int j = 0; j < a.nw; ++j) {
            CGState& c = a.cg[cell * a.nw + j];
            c.omega = ok ? 2.0 / (lo + hi) : 0.0;
            if (!ok && c.done == CG_RUNNING) c.done = CG_BREAKDOWN;
        }
        nd->extra[0] = lo;
        nd->extra[1] = hi;
    }
}

}  // namespace fftg
