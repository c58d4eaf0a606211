// Per-cell BDF controller: the step, error and order logic of one cell.
//
// It is written once over a "cell backend" C that owns the cell's vectors
// and Newton matrix (a thread per cell, or a group of lanes per cell in
// shared memory).  Every scalar here is uniform across the lanes serving
// the cell, so the group's control flow never diverges.
//
// Method (arXiv 2405.01713, Sec. 2): variable-order (1..5) variable-step
// BDF in Nordsieck form; accept a step iff ||E||_wrms < 1 (Eq. wrms, with
// weights from the previous step's solution); modified Newton on
// G(y) = y - gamma f(t_n, y) - a_n with the stopping test
// R ||delta_m|| < c_eps eps, R = max(c_r R, ||delta_m|| / ||delta_{m-1}||)
// (Eq. stop_newton).  Readings of points the paper leaves open:
//  * corrector coefficients l_j of Lambda(x) = prod_{i<=q} (1 + x/xi_i),
//    xi_i = (t_n - t_{n-i}) / h_n (variable-coefficient Nordsieck form);
//  * error estimate E = C_q Delta, C_q = 1/(1 + l_1 xi_{q+1});
//  * eps = 1/C_q (the correction may use c_eps of the error budget); R
//    starts at 1 in each Newton solve; at most 3 iterations; divergence
//    when a correction exceeds twice the previous one;
//  * the Newton matrix is rebuilt after 20 steps, when gamma moved by more
//    than 30 %, or after a failure; a stale matrix scales corrections by
//    2/(1 + gamma/gamma_M);
//  * step factors 1/((b ||E_p||)^(1/(p+1)) + 1e-6) in single precision,
//    biases 6/6/10 for orders q-1/q/q+1, threshold 1.5, caps 1e4 (first
//    step) / 10 / 1
//    (after a failure); order change considered after q+1 steps at q;
//  * failures: error test -> eta in [0.1, 0.9] (or order q-1), third
//    failure -> eta 0.1 at order 1 (reached by lowering the order of the
//    interpolating polynomial), seventh -> ERR_FAILURE;
//    Newton -> eta 0.25, tenth -> CONV_FAILURE;
//  * first step by the Hairer-Norsett-Wanner starting-step algorithm;
//  * each call is a cold start at order 1 that lands exactly on tout.
// All norms are kept squared (WRMS^2), so no square roots are taken.
#pragma once
#include "sunb_common.cuh"

namespace sunb {

// xi_i (i = 1..m) from h and previous step sizes: xi[i-1] = xi_i,
// inv[i-1] = 1/xi_i; entries from m on are 1 (unused).  The inverses come
// from one reciprocal (a batched inversion): with the running products
// P_i = xi[1] ... xi[i], 1/xi[i] = P_{i-1} / P_i, taken from 1/P_QMAX
// backwards.  Each carries a few roundings more than a division would, and
// the FP64 pipe, the kernels' bound, sees one reciprocal instead of m - 1.
__device__ __forceinline__ void bdf_xi(int m, double h, const double *hist, double *xi,
                                       double *inv)
{
    const double rh = rcp(h);
    double s = h, P[QMAX + 1];
    xi[0] = 1.0;
    inv[0] = 1.0;
    P[0] = 1.0;
#pragma unroll
    for (int i = 1; i < QMAX + 1; ++i) {
        double x = 1.0;
        if (i < m) {
            s += hist[i - 1];
            x = s * rh;
        }
        xi[i] = x;
        P[i] = P[i - 1] * x;
    }
    double R = rcp(P[QMAX]);              // 1 / (xi[1] ... xi[QMAX])
#pragma unroll
    for (int i = QMAX; i >= 1; --i) {
        inv[i] = R * P[i - 1];
        R *= xi[i];
    }
}

// Coefficients of prod_{i<q} (1 + x * inv[i]) -> l[0..q].
__device__ __forceinline__ void bdf_l(int q, const double *inv, double *l)
{
    l[0] = 1.0;
#pragma unroll
    for (int j = 1; j <= QMAX; ++j) l[j] = 0.0;
#pragma unroll
    for (int i = 0; i < QMAX; ++i) {
        if (i < q) {
#pragma unroll
            for (int j = QMAX; j >= 1; --j)
                if (j <= i + 1) l[j] += l[j - 1] * inv[i];
        }
    }
}

// a[k] for a runtime k in 0..QMAX, selected by predication: indexing a
// per-thread array with a runtime index would place the array in local
// memory, where the controller's few such reads cost a stack frame.
__device__ __forceinline__ double pick(const double *a, int k)
{
    double r = a[0];
#pragma unroll
    for (int j = 1; j <= QMAX; ++j)
        if (j == k) r = a[j];
    return r;
}

// 1/(p+1), p = 0..6
__constant__ float INV_P1F[7] = {1.0f, 1.0f / 2.0f, 1.0f / 3.0f, 1.0f / 4.0f, 1.0f / 5.0f, 1.0f / 6.0f,
                                 1.0f / 7.0f};

// Step factor eta_p = 1/((b ||E_p||)^(1/(p+1)) + 1e-6) from the squared WRMS
// norm d2 = ||E_p||^2, in single precision: L = log2(b ||E_p||) rounded to
// float, r = 2^(L/(p+1)), eta = 1/(r + 1e-6).  The factor is a heuristic
// that only scales h; the decisions it makes (keep h below 1.5, the order of
// the largest factor) are taken in this precision, and the oracle takes them
// in the same one.  L = log2 b + (e + log2 m)/2 for d2 = 2^e m, e and the
// leading 23 bits of m read from the double's bits: the whole double range
// without an FP64 instruction (the FP64 pipe is the kernels' bound; the
// float functions run on the FP32 pipe).  d2 = 0 or subnormal gives L = -inf
// (eta = 1e6, above every growth cap), d2 = inf gives L = +inf (eta = 0).
__device__ __forceinline__ double eta_from(double d2, int p, float bias)
{
    const int hi = __double2hiint(d2);
    float L;
    if (hi >= 0x7ff00000) {
        L = __int_as_float(0x7f800000);
    } else if (hi < 0x00100000) {
        L = -__int_as_float(0x7f800000);
    } else {
        const int e = (hi >> 20) - 1023;
        const float m = __int_as_float(0x3f800000 | ((hi & 0x000fffff) << 3) |
                                       (int)((unsigned)__double2loint(d2) >> 29));   // [1, 2)
        L = fmaf(0.5f, (float)e + log2f(m), log2f(bias));
    }
    const float r = exp2f(L * INV_P1F[p]);
    return (double)(1.0f / (r + 1e-6f));
}

// sum_{i<q-1} inv[i] and prod_{i<q-1} xi[i] (the order q-1 estimate's
// coefficients), by predication over the unrolled range
__device__ __forceinline__ void lower_order_sums(int q, const double *inv, const double *xi, double &l1m,
                                                 double &pm)
{
    l1m = 0.0;
    pm = 1.0;
#pragma unroll
    for (int i = 0; i < QMAX - 1; ++i)
        if (i < q - 1) { l1m += inv[i]; pm *= xi[i]; }
}

// Coefficients e of x * prod_{i<q-1} (x + nodes[i]) (e[j] multiplies x^(j+1)).
__device__ __forceinline__ void decrease_coeffs(int q, const double *nodes, double *e)
{
    e[0] = 1.0;
#pragma unroll
    for (int j = 1; j <= QMAX; ++j) e[j] = 0.0;
#pragma unroll
    for (int i = 0; i < QMAX - 1; ++i) {
        if (i < q - 1) {
#pragma unroll
            for (int j = QMAX; j >= 1; --j)
                if (j <= i + 1) e[j] = e[j - 1] + e[j] * nodes[i];
            e[0] *= nodes[i];
        }
    }
}

// Equal-step coefficients (xi_i = i): l = coefficients of prod (1 + x/i),
// the classical fixed-step Nordsieck BDF vectors.  Used whenever the last q
// steps had the current size, so the coefficients need no divisions.
__constant__ double GEAR_L[QMAX + 1][QMAX + 1] = {
    {1.0, 0, 0, 0, 0, 0},
    {1.0, 1.0, 0, 0, 0, 0},
    {1.0, 3.0 / 2.0, 1.0 / 2.0, 0, 0, 0},
    {1.0, 11.0 / 6.0, 1.0, 1.0 / 6.0, 0, 0},
    {1.0, 25.0 / 12.0, 35.0 / 24.0, 5.0 / 12.0, 1.0 / 24.0, 0},
    {1.0, 137.0 / 60.0, 15.0 / 8.0, 17.0 / 24.0, 1.0 / 8.0, 1.0 / 120.0}};

__constant__ double GEAR_INV[QMAX + 1] = {1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0};
// 1/l_1 = 1/H_q (H_q harmonic numbers) and C_q = 1/(1 + H_q (q+1))
__constant__ double GEAR_IL1[QMAX + 1] = {1.0, 1.0, 2.0 / 3.0, 6.0 / 11.0, 12.0 / 25.0, 60.0 / 137.0};
__constant__ double GEAR_CQ[QMAX + 1] = {1.0, 1.0 / 3.0, 2.0 / 11.0, 6.0 / 50.0, 12.0 / 137.0, 60.0 / 882.0};

// The first steps of a cell for the explicit controller, the same as
// CellRun::begin_body's: y0 into V_Z0, f(t0, y0) into V_F, the weights from
// y0, and the starting step h of Hairer, Norsett & Wanner (order 1, WRMS
// norms), at most tout - t0.  False when the cell is finished already:
// tout <= t0, or a non-finite y0 or f (s.status = ST_NONFINITE).  (The BDF
// keeps its inline copy: calling this from begin_body changed the register
// allocation of the thread-per-cell BDF kernel.)
template <class C>
__device__ __forceinline__ bool start_cell(C &c, const Controls &ctl, CellStats &s, double &h)
{
    const double t0 = ctl.t0, tout = ctl.tout;
    c.load_y(V_Z0);
    if (!(tout > t0)) return false;
    c.rhs_start(V_Z0, V_F);
    s.nfe++;
    if (!c.all_finite(V_F) || !c.all_finite(V_Z0)) {
        s.status = ST_NONFINITE;
        return false;
    }
    c.set_weights(V_Z0, ctl.rtol);
    const double span = tout - t0;
    const double d0 = c.wrms2(V_Z0), d1 = c.wrms2(V_F);   // squared
    double h0 = (d0 < 1e-10 || d1 < 1e-10) ? 1e-6 * span : 0.01 * sqrt(d0 * rcp(d1));
    if (h0 > span) h0 = span;
    c.axpby(V_Y, 1.0, V_Z0, h0, V_F);
    c.rhs_start(V_Y, V_DEL);
    s.nfe++;
    const double rh0 = rcp(h0);
    const double d2 = c.wrms2_lin(rh0, V_DEL, -rh0, V_F);
    const double dm = fmax(d1, d2);
    double h1 = (dm <= 1e-30) ? fmax(1e-6 * span, h0 * 1e-3) : sqrt(0.01 * rcp(sqrt(dm)));
    h = fmin(100.0 * h0, h1);
    if (!(h > 0.0)) h = 1e-6 * span;
    h = fmin(h, span);
    return true;
}

// The controller as a state machine that advances a cell by at most one
// step attempt (or, for backends that ask for it, one Newton iteration) per
// call ("superstep").  Its phases -- STEP (start a step),
// ATTEMPT (predict, coefficients), SETUP (f and the Newton matrix at the
// prediction), NEWTON (the iterations: f, solve, convergence test) and POST
// (Newton failure, error test, accept, step and order selection) -- are
// visited in this fixed order inside a superstep.  Cells that share a warp
// (a thread per cell, or several lane groups per warp) therefore run the
// right-hand-side call of NEWTON, the set-up call of SETUP and the control
// logic together, whatever their step counts, instead of diverging through
// nested loops.  A cell's arithmetic is exactly that of the sequential
// algorithm (bdf_cell below runs it sequentially).
enum Phase : int {
    // the two f evaluations of a cell's start, for backends with
    // C::kFoldedStart (CellRun::begin_folded); below PH_STEP
    PH_START0 = -2, PH_START1 = -1,
    PH_STEP = 0, PH_ATTEMPT = 1, PH_SETUP = 2, PH_NEWTON = 3, PH_POST = 4,
    PH_DONE = 5,    // finished; the caller collects s and may begin another cell
    PH_EXIT = 6     // no cell left for this thread or group (set by run_cells)
};

template <class C>
struct CellRun {
    int phase;
    CellStats s;
    int qmax;
    // integration state
    double tout, t, h, gamma_M, etamax, h_ks;
    double hist[QMAX + 1];
    int q, qwait, have_M, force_setup, nst_lastsetup, have_ks, nsame;
    // current step / attempt
    int last, ncf, nef;
    double dsm2, Cq, il1, gamma;
    double etaq, emq;     // the order-q and order-(q-1) step factors of the attempt
                          // (backends with C::kSharedEtaQ; emq 0 where not needed)
    double l[QMAX + 1], xi[QMAX + 1], inv[QMAX + 1];
    // current Newton solve
    int fresh, conv, setup_now, m;
    double delp2, R2, cstale;

    __device__ void finish(C &c)
    {
        s.qlast = q;
        c.store_y(V_Z0);
        phase = PH_DONE;
    }

    // first steps of a cell: load, f(t0, y0), weights, starting step size.
    // Backends that ask for it (C::kOutlineRare) run this and the failure
    // paths out of line, so that the kernel's hot loop carries less code
    // (instruction fetch is one of the lane-group kernel's leading stalls);
    // for thread-per-cell cells they are too frequent to pay a call.
    __device__ __forceinline__ void begin(C &c, const Controls &ctl)
    {
        if constexpr (C::kFoldedStart) begin_folded(c, ctl);
        else if constexpr (C::kOutlineRare) begin_outlined(c, ctl);
        else begin_body(c, ctl);
    }

    // Backends with C::kFoldedStart (a thread per cell, where the cells of a
    // warp begin at different supersteps): the start's two f evaluations
    // run at the Newton iterations' f call site, in phases START0 and
    // START1, so that a beginning cell joins its warp's evaluations instead
    // of running its own while the other 31 lanes wait.  The arithmetic is
    // begin_body's: f(t0, y0) arrives in V_F and is kept in V_ACOR while
    // f(t0 + h0, y0 + h0 f0) arrives in V_F; between the phases h holds h0
    // and delp2 holds ||f0||^2 (both unused until the first step).
    __device__ __forceinline__ void begin_folded(C &c, const Controls &ctl)
    {
        tout = ctl.tout;
        qmax = ctl.max_order < 1 ? 1 : (ctl.max_order > QMAX ? QMAX : ctl.max_order);
        s.nst = s.nfe = s.nje = s.nni = s.ncf = s.nef = 0;
        s.qlast = 1;
        s.status = ST_SUCCESS;
        q = 1;
        c.load_y(V_Z0);
        if (!(tout > ctl.t0)) { finish(c); return; }
        c.newton_init();           // V_Y = y0
        setup_now = 0;
        phase = PH_START0;
    }
    __device__ __forceinline__ void start_after_f(C &c, const Controls &ctl)
    {
        const double t0 = ctl.t0, span = tout - t0;
        if (phase == PH_START0) {   // V_F = f(t0, y0)
            if (!c.all_finite(V_F) || !c.all_finite(V_Z0)) {
                s.status = ST_NONFINITE;
                finish(c);
                return;
            }
            c.set_weights(V_Z0, ctl.rtol);
            const double d0 = c.wrms2(V_Z0), d1 = c.wrms2(V_F);   // squared
            double h0 = (d0 < 1e-10 || d1 < 1e-10) ? 1e-6 * span : 0.01 * sqrt(d0 * rcp(d1));
            if (h0 > span) h0 = span;
            c.axpby(V_Y, 1.0, V_Z0, h0, V_F);
            c.copy(V_ACOR, V_F);
            h = h0;
            delp2 = d1;
            phase = PH_START1;
            return;
        }
        // V_F = f(t0 + h0, y0 + h0 f0), V_ACOR = f0
        const double h0 = h, d1 = delp2;
        const double rh0 = rcp(h0);
        const double d2 = c.wrms2_lin(rh0, V_F, -rh0, V_ACOR);
        const double dm = fmax(d1, d2);
        double h1 = (dm <= 1e-30) ? fmax(1e-6 * span, h0 * 1e-3) : sqrt(0.01 * rcp(sqrt(dm)));
        h = fmin(100.0 * h0, h1);
        if (!(h > 0.0)) h = 1e-6 * span;
        h = fmin(h, span);
        c.scale(V_Z1, h, V_ACOR);
        c.rec_init(h);
        t = t0;
        qwait = 2; have_M = 0; force_setup = 1; nst_lastsetup = 0; have_ks = 0; nsame = 0;
#pragma unroll
        for (int i = 0; i <= QMAX; ++i) hist[i] = 0.0;
        gamma_M = 0.0; etamax = ETA_MAX_FIRST; h_ks = 0.0;
        phase = PH_STEP;
    }
    __device__ __noinline__ void begin_outlined(C &c, const Controls &ctl) { begin_body(c, ctl); }
    __device__ __forceinline__ void begin_body(C &c, const Controls &ctl)
    {
        const double t0 = ctl.t0;
        tout = ctl.tout;
        qmax = ctl.max_order < 1 ? 1 : (ctl.max_order > QMAX ? QMAX : ctl.max_order);
        s.nst = s.nfe = s.nje = s.nni = s.ncf = s.nef = 0;
        s.qlast = 1;
        s.status = ST_SUCCESS;
        q = 1;
        c.load_y(V_Z0);
        if (!(tout > t0)) { finish(c); return; }
        c.rhs_start(V_Z0, V_F);
        s.nfe++;
        if (!c.all_finite(V_F) || !c.all_finite(V_Z0)) {
            s.status = ST_NONFINITE;
            finish(c);
            return;
        }
        c.set_weights(V_Z0, ctl.rtol);
        // starting step (Hairer, Norsett & Wanner, order 1)
        {
            const double span = tout - t0;
            const double d0 = c.wrms2(V_Z0), d1 = c.wrms2(V_F);   // squared
            double h0 = (d0 < 1e-10 || d1 < 1e-10) ? 1e-6 * span : 0.01 * sqrt(d0 * rcp(d1));
            if (h0 > span) h0 = span;
            c.axpby(V_Y, 1.0, V_Z0, h0, V_F);
            c.rhs_start(V_Y, V_DEL);
            s.nfe++;
            const double rh0 = rcp(h0);
            const double d2 = c.wrms2_lin(rh0, V_DEL, -rh0, V_F);
            const double dm = fmax(d1, d2);
            double h1 = (dm <= 1e-30) ? fmax(1e-6 * span, h0 * 1e-3) : sqrt(0.01 * rcp(sqrt(dm)));
            h = fmin(100.0 * h0, h1);
            if (!(h > 0.0)) h = 1e-6 * span;
            h = fmin(h, span);
        }
        c.scale(V_Z1, h, V_F);
        c.rec_init(h);
        t = t0;
        qwait = 2; have_M = 0; force_setup = 1; nst_lastsetup = 0; have_ks = 0; nsame = 0;
#pragma unroll
        for (int i = 0; i <= QMAX; ++i) hist[i] = 0.0;
        gamma_M = 0.0; etamax = ETA_MAX_FIRST; h_ks = 0.0;
        phase = PH_STEP;
    }

    __device__ void start_newton(C &c)
    {
        c.newton_init();
        delp2 = 0.0;
        R2 = 1.0;
        // 2/(1 + gamma/gamma_M) with one reciprocal
        cstale = (gamma != gamma_M) ? 2.0 * gamma_M * rcp(gamma_M + gamma) : 1.0;
        m = 0;
        phase = PH_NEWTON;
    }

    __device__ void superstep(C &c, const Controls &ctl)
    {
        if (phase == PH_STEP) {
            if (!(t < tout)) {
                finish(c);
            } else if (s.nst >= ctl.max_steps) {
                s.status = ST_TOO_MUCH_WORK;
                finish(c);
            } else {
                last = 0;
                if (t + h >= tout || tout - (t + h) <= 4.0 * 2.220446049250313e-16 * fabs(tout)) {
                    const double hn = tout - t;
                    c.rescale(q, hn * rcp(h));
                    h = hn;
                    last = 1;
                    nsame = 0;
                }
                c.set_weights(V_Z0, ctl.rtol);          // Eq. wrms: weights from y^{n-1}
                ncf = 0;
                nef = 0;
                phase = PH_ATTEMPT;
            }
        }
        if (phase == PH_ATTEMPT) {
            c.predict(q);
            if (nsame >= q) {
#pragma unroll
                for (int i = 0; i <= QMAX; ++i) {
                    xi[i] = (double)(i + 1);
                    inv[i] = GEAR_INV[i];
                    l[i] = GEAR_L[q][i];
                }
                il1 = GEAR_IL1[q];
                Cq = GEAR_CQ[q];
            } else {
                bdf_xi(q + 1, h, hist, xi, inv);
                bdf_l(q, inv, l);
                // 1/l_1 and C_q = 1/(1 + l_1 xi_{q+1}) from one reciprocal
                const double cq1 = 1.0 + l[1] * pick(xi, q);
                const double r = rcp(l[1] * cq1);
                il1 = r * cq1;
                Cq = r * l[1];
            }
            gamma = h * il1;
            fresh = 0;
            setup_now = 0;
            if constexpr (C::kKrylov) {   // matrix-free: nothing to build or keep
                have_M = 1; fresh = 1; gamma_M = gamma;
                start_newton(c);
            } else {
                if (force_setup || !have_M || s.nst >= nst_lastsetup + MSBP ||
                    fabs(gamma - gamma_M) > DGMAX * gamma_M)        // |gamma/gamma_M - 1| > DGMAX
                    phase = PH_SETUP;
                else
                    start_newton(c);
            }
        }
        // the Newton matrix at the prediction z0: built by the first Newton
        // iteration below, whose f evaluation is at y = z0.  A backend whose
        // set-up scratch is taken by another cell of the warp defers the
        // set-up to the next superstep.
        if (phase == PH_SETUP && c.acquire_setup()) {
            s.nje++;
            gamma_M = gamma; nst_lastsetup = s.nst; fresh = 1; force_setup = 0;
            setup_now = 1;
            start_newton(c);
        }
        // modified Newton iterations (Eq. stop_newton) until convergence,
        // divergence or MAXCOR, at most C::kNewtonPerSuperstep of them in
        // this superstep; a cell that needs more continues in the next
        // superstep, at the same f call site as the other cells' first
        // iterations (the arithmetic does not depend on where it stops)
        // (with C::kFoldedStart the same f call serves the start phases)
        int iters_here = 0;
        while (phase == PH_NEWTON || (C::kFoldedStart && phase < 0)) {
            const int ok = c.newton_f(setup_now != 0, gamma);
            s.nfe++;
            if constexpr (C::kFoldedStart) {
                if (phase < 0) {
                    start_after_f(c, ctl);
                    if (++iters_here >= C::kNewtonPerSuperstep) break;
                    continue;
                }
            }
            if (setup_now) s.nfe += c.f_per_setup();
            if (setup_now) { have_M = ok; setup_now = 0; }
            bool done = false;
            conv = 0;
            if (!have_M) {
                done = true;                                 // singular matrix
            } else {
                s.nni++;
                c.newton_residual(h, il1);
                // backends with C::kKrylov: the inexact Newton iteration's GMRES
                // solve, whose f evaluations count here
                if constexpr (C::kKrylov) s.nfe += c.solve_krylov(gamma, Cq);
                else c.solve(V_DEL);
                const double dn2 = c.newton_update(cstale);
                if (!(dn2 <= 1.7e308)) {
                    done = true;                             // not finite
                } else {
                    if (m > 0) R2 = fmax(CRDOWN * CRDOWN * R2, dn2 * rcp(delp2));
                    if (R2 * dn2 * (Cq * Cq) < NLS_COEF * NLS_COEF) { conv = 1; done = true; }
                    else if (m + 1 == MAXCOR || (m > 0 && dn2 > RDIV * RDIV * delp2)) done = true;
                    else { delp2 = dn2; ++m; }
                }
            }
            if (done) phase = PH_POST;
            if (++iters_here >= C::kNewtonPerSuperstep) break;
        }
        if (phase == PH_POST) post(c);
    }

    __device__ void post(C &c)
    {
        if (!conv && !fresh) {        // stale matrix: rebuild at the predicted state and retry
            phase = PH_SETUP;
            return;
        }
        if (!conv) {                  // Newton failure
            if constexpr (C::kOutlineRare) fail_newton_outlined(c);
            else fail_newton(c);
            return;
        }
        dsm2 = (Cq * Cq) * c.wrms2(V_ACOR);
        // Backends with C::kSharedEtaQ (a warp of 32 thread-per-cell cells):
        // the cells reach the error test together, and both the failing
        // ones and the growing ones need the order-q factor; one evaluation
        // here, before the branch, takes one pass of the warp instead of
        // one per path (same value: same function of the same arguments).
        if constexpr (C::kSharedEtaQ) {
            etaq = eta_from(dsm2, q, BIAS_Q);
            // likewise the order q-1 factor, which the first two error-test
            // failures of a step and the order selection that comes due
            // after an accepted step both need (the failures from the
            // predicted z_q, which the prediction leaves unchanged, the
            // selection from the corrected z_q + l_q Delta)
            emq = 0.0;
            if (q > 1) {
                const bool fail = dsm2 >= 1.0;
                if (fail ? (nef + 1 < MXNEF1) : (!last && qwait == 1)) {
                    double l1m, pm;
                    lower_order_sums(q, inv, xi, l1m, pm);
                    const double f = pm * rcp(l1m);
                    const double d2 = (fail ? c.wrms2(q) : c.wrms2_corrected(q, pick(l, q))) * f * f;
                    emq = eta_from(d2, q - 1, BIAS_QM1);
                }
            }
        }
        Tail tl;
        if (dsm2 >= 1.0) {            // error-test failure (accept iff ||LTE|| < 1)
            if constexpr (C::kOutlineRare) fail_error_outlined(c, tl);
            else fail_error(c, tl);
        } else {
            accept_step(c, tl);
        }
        if constexpr (C::kSharedEtaQ) end_attempt(c, tl);
    }

    // The common end of an error-test failure and an accepted step, for
    // backends with C::kSharedEtaQ, whose warps nearly always hold cells on
    // both paths: the paths record an order decrease from order dec (0:
    // none) and a rescale by eta (1: none), and end_attempt applies them
    // once after the branch, in the order the paths would (decrease, then
    // h *= eta and the rescale at the new order), then the step-size
    // underflow check of a failure.  Other backends apply them in the paths.
    struct Tail {
        int dec = 0, fail = 0;
        double eta = 1.0;
    };
    __device__ __forceinline__ void end_attempt(C &c, const Tail &tl)
    {
        if (tl.dec) {
            // the nodes of the polynomial the decrease keeps: xi_i after an
            // accepted step; after a failure (t_n - t_{n-1-i})/h_n, the sums
            // of the previous steps, = xi_{i+1} - 1 of the failed attempt
            double nodes[QMAX], e[QMAX + 1];
#pragma unroll
            for (int i = 0; i < QMAX - 1; ++i) nodes[i] = tl.fail ? xi[i + 1] - 1.0 : xi[i];
            nodes[QMAX - 1] = 0.0;                 // (decrease_coeffs reads i < q - 1)
            decrease_coeffs(tl.dec, nodes, e);
            c.order_decrease(tl.dec, e);
        }
        if (tl.eta != 1.0) {
            h *= tl.eta;
            c.rescale(q, tl.eta);
            if (tl.fail && t + h == t) { s.status = ST_H_TOO_SMALL; finish(c); }
        }
    }

    // the rarer outcomes of an attempt (out of line for C::kOutlineRare)
    __device__ __noinline__ void fail_newton_outlined(C &c) { fail_newton(c); }
    __device__ __noinline__ void fail_error_outlined(C &c, Tail &tl) { fail_error(c, tl); }
    __device__ __forceinline__ void fail_newton(C &c)
    {
        c.unpredict(q);
        s.ncf++; ncf++;
        if (ncf >= MXNCF) { s.status = ST_CONV_FAILURE; finish(c); return; }
        h *= ETA_CF;
        c.rescale(q, ETA_CF);
        force_setup = 1; etamax = 1.0; last = 0; nsame = 0;
        if (t + h == t) { s.status = ST_H_TOO_SMALL; finish(c); return; }
        phase = PH_ATTEMPT;
    }

    __device__ __forceinline__ void fail_error(C &c, Tail &tl)
    {
        {
            c.unpredict(q);
            s.nef++; nef++;
            if (nef >= MXNEF) { s.status = ST_ERR_FAILURE; finish(c); return; }
            if (nef < MXNEF1) {
                double eta;
                if constexpr (C::kSharedEtaQ) eta = etaq;
                else eta = eta_from(dsm2, q, BIAS_Q);
                int newq = q;
                if (q > 1) {
                    double em;
                    if constexpr (C::kSharedEtaQ) {
                        em = emq;
                    } else {
                        double l1m, pm;
                        lower_order_sums(q, inv, xi, l1m, pm);
                        const double f = pm * rcp(l1m);
                        em = eta_from(c.wrms2(q) * f * f, q - 1, BIAS_QM1);
                    }
                    if (em > eta) { eta = em; newq = q - 1; }
                }
                eta = fmin(ETA_MAX_EF, fmax(ETA_MIN_EF, eta));
                if (newq < q) {
                    if constexpr (C::kSharedEtaQ) {
                        tl.dec = q;
                    } else {
                        double nodes[QMAX], sacc = 0.0, e[QMAX + 1];
                        const double rh = rcp(h);
                        for (int i = 0; i < QMAX; ++i) {
                            sacc += hist[i];
                            nodes[i] = sacc * rh;
                        }
                        decrease_coeffs(q, nodes, e);
                        c.order_decrease(q, e);
                    }
                    q = newq; qwait = q + 1;
                }
                if constexpr (C::kSharedEtaQ) {
                    tl.eta = eta;
                } else {
                    h *= eta;
                    c.rescale(q, eta);
                }
            } else {
                // third failure on: order 1 through the interpolating
                // polynomials (keeps the line through the last two accepted
                // states), eta = 0.1
                if (q > 1) {
                    double nodes[QMAX], sacc = 0.0, e[QMAX + 1];
                    const double rh = rcp(h);
                    for (int i = 0; i < QMAX; ++i) {
                        sacc += hist[i];
                        nodes[i] = sacc * rh;
                    }
                    for (; q > 1; --q) {
                        decrease_coeffs(q, nodes, e);
                        c.order_decrease(q, e);
                    }
                }
                if constexpr (C::kSharedEtaQ) {
                    tl.eta = ETA_MIN_EF;
                } else {
                    h *= ETA_MIN_EF;
                    c.rescale(q, ETA_MIN_EF);
                }
                qwait = 2; have_ks = 0;
            }
            etamax = 1.0; last = 0; nsame = 0;
            phase = PH_ATTEMPT;
            if constexpr (C::kSharedEtaQ) {
                tl.fail = 1;        // end_attempt rescales, then checks h
            } else {
                if (t + h == t) { s.status = ST_H_TOO_SMALL; finish(c); return; }
            }
        }
    }

    __device__ __forceinline__ void accept_step(C &c, Tail &tl)
    {
        s.nst++;
        t = last ? tout : t + h;
        c.correct(q, l);
#pragma unroll
        for (int i = QMAX; i > 0; --i) hist[i] = hist[i - 1];
        hist[0] = h;
        if (last) {
            c.rec_accept(q, q, l, 0.0, gamma, il1, h, ncf, nef);
            finish(c);
            return;
        }
        qwait--;
        const double l1 = l[1];
        double eta = 1.0;
        int newq = q;
        const double inv_q = pick(inv, q);
        const double kfac = l1 * pick(l, q) * Cq;     // h^{q+1} y^{(q+1)}/(q+1)! = kfac * Delta
        if constexpr (C::kSharedEtaQ) eta = etaq;
        else eta = eta_from(dsm2, q, BIAS_Q);
        if (qwait == 0) {
            double em = 0.0, ep = 0.0;
            if (q > 1) {
                if constexpr (C::kSharedEtaQ) {
                    em = emq;
                } else {
                    double l1m, pm;
                    lower_order_sums(q, inv, xi, l1m, pm);
                    const double f = pm * rcp(l1m);
                    const double d2 = c.wrms2(q) * f * f;
                    em = eta_from(d2, q - 1, BIAS_QM1);
                }
            }
            if (q < qmax && have_ks) {
                double rq = 1.0;
                const double rr = h * rcp(h_ks);
                for (int i = 0; i <= q; ++i) rq *= rr;
                double pp = 1.0;
#pragma unroll
                for (int i = 0; i <= QMAX; ++i)
                    if (i <= q) pp *= xi[i];
                const double l1p = l1 + inv_q;
                const double f = pp * rcp(l1p * (q + 2));
                const double d2 = c.wrms2_lin(kfac, V_ACOR, -rq, V_KS) * f * f;
                ep = eta_from(d2, q + 1, BIAS_QP1);
            }
            if (em > eta && em >= ep) { eta = em; newq = q - 1; }
            else if (ep > eta) { eta = ep; newq = q + 1; }
        }
        if (eta < ETA_THRESH) { eta = 1.0; newq = q; }
        else eta = fmin(eta, etamax);
        c.rec_accept(q, newq == q + 1 ? q + 1 : q, l, inv_q, gamma, il1, h, ncf, nef);
        if (newq == q + 1) c.order_increase(q, l, inv_q);
        else if (newq == q - 1) {
            if constexpr (C::kSharedEtaQ) {
                tl.dec = q;
            } else {
                double e[QMAX + 1];
                decrease_coeffs(q, xi, e);
                c.order_decrease(q, e);
            }
        }
        if (newq != q || qwait == 0) { q = newq; qwait = q + 1; have_ks = 0; }
        if (qwait == 1 && q < qmax) {
            c.scale(V_KS, kfac, V_ACOR);
            h_ks = h; have_ks = 1;
        }
        if (eta != 1.0) {
            if constexpr (C::kSharedEtaQ) {
                tl.eta = eta;
            } else {
                h *= eta;
                c.rescale(q, eta);
            }
            nsame = 0;
        } else if (nsame < QMAX) {
            ++nsame;
        }
        etamax = ETA_MAX;
        phase = PH_STEP;
    }
};

// One cell from start to finish (the sequential use of the state machine).
template <class C>
__device__ void bdf_cell(C &c, const Controls &ctl, CellStats &s)
{
    CellRun<C> run;
    run.begin(c, ctl);
    while (run.phase != PH_DONE) run.superstep(c, ctl);
    s = run.s;
}

// Runs the cells handed out by next() (a cell index, or -1 when none is
// left) on this thread or lane group, one superstep at a time: a thread
// (group) whose cell finishes begins its next cell at once while the rest
// of its warp keeps stepping.  wmask holds the warp's launched threads; the
// loop ends when none of them has a cell left.  bind(cell) points the
// backend at a cell before it begins; done(cell, stats) reports it.
// Run is the controller (CellRun, or ErkRun for the explicit method).
template <template <class> class Run = CellRun, class C, class Next, class Bind, class Done>
__device__ __forceinline__ void run_cells(C &c, const Controls &ctl, unsigned wmask, Next next,
                                          Bind bind, Done done)
{
    Run<C> run;
    run.phase = PH_DONE;
    long long cell = -1;
    for (;;) {
        if (run.phase == PH_DONE) {
            cell = next();
            if (cell >= 0) {
                bind(cell);
                run.begin(c, ctl);
            } else {
                run.phase = PH_EXIT;
            }
        }
        if (__all_sync(wmask, run.phase == PH_EXIT)) break;
        if (run.phase < PH_DONE) run.superstep(c, ctl);
        if (run.phase == PH_DONE) done(cell, run.s);
    }
}

// Mask of the launched threads of the calling thread's warp.
__device__ __forceinline__ unsigned launched_warp_mask()
{
    const int first = (int)(threadIdx.x & ~31u);
    const int n = min(32, (int)blockDim.x - first);
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

}  // namespace sunb
