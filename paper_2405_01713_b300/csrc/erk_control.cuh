// Explicit Runge-Kutta controller: the explicit alternative to the BDF
// (arXiv 2405.01713, Sec. 4.1.5), a fourth-order, adaptive-step method of
// the ARKODE kind whose step adaptivity rests on an embedded estimate of
// the local error under the same WRMS test as the BDF (Sec. 2, Eq. wrms).
// The paper names no table; this is Merson's five-stage pair, order 4 with
// an embedded order-3 solution (Merson 1957; Hairer, Norsett & Wanner,
// Solving ODEs I, II.4):
//   k_j = f(y_n + h sum_{m<j} a_jm k_m),  y_{n+1} = y_n + h sum b_j k_j,
//   E = h sum (b_j - bh_j) k_j,  accept iff ||E||_wrms < 1, weights from y_n;
// step factor 0.9 (1/||E||)^(1/4), at most 10 after an accepted step (1e4
// after the first), at most 1 after a rejection, at most 0.3 from the second
// rejection of a step on, at least 0.1; seven rejections of one step give
// ERR_FAILURE.  The starting step is the BDF's (start_cell); the last step
// lands exactly on tout; k_1 = f(y_n) is kept across a rejection.
//
// The backend keeps the stage derivatives k_0..k_4 in vector slots 1..5
// (the Nordsieck columns, which the explicit method does not use) and
// provides erk_stage (V_Y = V_Z0 + h sum_{m<j} a_jm k_m), erk_rhs (k_j =
// f(V_Y)), erk_error2 (||E||^2) and erk_accept (V_Z0 += h sum b_m k_m).
#pragma once
#include "bdf_control.cuh"

namespace sunb {

// Merson's table (runtime stage index j: constant memory)
static __constant__ double ERK_A[5][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {1.0 / 3.0, 0.0, 0.0, 0.0},
    {1.0 / 6.0, 1.0 / 6.0, 0.0, 0.0},
    {1.0 / 8.0, 0.0, 3.0 / 8.0, 0.0},
    {1.0 / 2.0, 0.0, -3.0 / 2.0, 2.0},
};
static __constant__ double ERK_B[5] = {1.0 / 6.0, 0.0, 0.0, 2.0 / 3.0, 1.0 / 6.0};
static __constant__ double ERK_BH[5] = {1.0 / 10.0, 0.0, 3.0 / 10.0, 2.0 / 5.0, 1.0 / 5.0};

constexpr double ERK_SAFETY = 0.9;
constexpr double ERK_ETA_MAX = 10.0;      // growth cap after an accepted step (1e4 after the first)
constexpr double ERK_ETA_MIN = 0.1;       // least factor after a rejection
constexpr double ERK_ETA_MAX_NEF = 0.3;   // cap from the second rejection of a step on

// One attempt per superstep: its five stages run in a loop around one f
// call site, so the cells of a warp evaluate f together whatever their
// step counts.
template <class C>
struct ErkRun {
    int phase;
    CellStats s;
    double tout, t, h, etamax;
    int nef, have_k1;

    __device__ void finish(C &c)
    {
        s.qlast = 4;
        c.store_y(V_Z0);
        phase = PH_DONE;
    }

    __device__ __forceinline__ void begin(C &c, const Controls &ctl)
    {
        tout = ctl.tout;
        s.nst = s.nfe = s.nje = s.nni = s.ncf = s.nef = 0;
        s.status = ST_SUCCESS;
        if (!start_cell(c, ctl, s, h)) { finish(c); return; }
        c.scale(1, 1.0, V_F);                 // k_0 = f(y0)
        have_k1 = 1;
        t = ctl.t0;
        nef = 0;
        etamax = ETA_MAX_FIRST;
        phase = PH_STEP;
    }

    __device__ void superstep(C &c, const Controls &ctl)
    {
        if (!(t < tout)) { finish(c); return; }
        if (s.nst >= ctl.max_steps) { s.status = ST_TOO_MUCH_WORK; finish(c); return; }
        bool last = false;
        if (t + h >= tout || tout - (t + h) <= 4.0 * 2.220446049250313e-16 * fabs(tout)) {
            h = tout - t;
            last = true;
        }
        c.set_weights(V_Z0, ctl.rtol);
        for (int j = have_k1 ? 1 : 0; j < 5; ++j) {
            c.erk_stage(j, h);
            c.erk_rhs(j);
            s.nfe++;
        }
        have_k1 = 1;
        const double e2 = c.erk_error2(h);   // ||E||_wrms^2
        if (e2 < 1.0) {                      // accept
            c.erk_accept(h);
            t = last ? tout : t + h;
            s.nst++;
            have_k1 = 0;
            nef = 0;
            if (last) { finish(c); return; }
            const double eta = e2 > 0.0 ? ERK_SAFETY / sqrt(sqrt(sqrt(e2))) : etamax;
            h *= fmin(eta, etamax);
            etamax = ERK_ETA_MAX;
            return;
        }
        s.nef++;                             // reject (a non-finite E counts as one)
        if (++nef >= MXNEF) { s.status = ST_ERR_FAILURE; finish(c); return; }
        double eta = (e2 <= 1.7e308) ? ERK_SAFETY / sqrt(sqrt(sqrt(e2))) : ERK_ETA_MIN;
        if (nef >= 2) eta = fmin(eta, ERK_ETA_MAX_NEF);
        h *= fmax(ERK_ETA_MIN, eta);
        etamax = 1.0;
        if (t + h == t) { s.status = ST_H_TOO_SMALL; finish(c); }
    }
};

}  // namespace sunb
