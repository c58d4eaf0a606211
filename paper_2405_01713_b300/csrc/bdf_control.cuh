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
//  * step factors 1/((b ||E_p||)^(1/(p+1)) + 1e-6), biases 6/6/10 for
//    orders q-1/q/q+1, threshold 1.5, caps 1e4 (first step) / 10 / 1
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

// xi_i (i = 1..m) from h and previous step sizes; inv[i-1] = 1/xi_i.
__device__ __forceinline__ void bdf_xi(int m, double h, const double *hist, double *xi,
                                       double *inv)
{
    const double rh = rcp(h);
    double s = h;
    xi[0] = 1.0;
    inv[0] = 1.0;
#pragma unroll
    for (int i = 1; i < QMAX + 1; ++i) {
        if (i < m) {
            s += hist[i - 1];
            xi[i] = s * rh;
            inv[i] = h * rcp(s);
        }
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

// Step factor from a squared WRMS error norm at order p.
__device__ __forceinline__ double eta_from(double d2, int p, double bias)
{
    const double inv_p1[7] = {1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0};
    // (bias * sqrt(d2))^(1/(p+1)) = exp(0.5 * log(bias^2 d2) / (p+1))
    double r = exp(0.5 * log(bias * bias * d2) * inv_p1[p]);
    return rcp(r + 1e-6);
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

// eta_p >= 1.5 exactly when bias^2 * ||E_p||^2 <= (2/3 - 1e-6)^(2(p+1)):
// the step-size choice takes the power only when a change can follow.
__device__ __forceinline__ double eta_viable2(int p)
{
    const double b = 2.0 / 3.0 - 1e-6;
    double r = 1.0;
    for (int i = 0; i < 2 * (p + 1); ++i) r *= b;
    return r;
}

template <class C>
__device__ void bdf_cell(C &c, const Controls &ctl, CellStats &s)
{
    const double t0 = ctl.t0, tout = ctl.tout;
    const int qmax = ctl.max_order < 1 ? 1 : (ctl.max_order > QMAX ? QMAX : ctl.max_order);
    s.nst = s.nfe = s.nje = s.nni = s.ncf = s.nef = 0;
    s.qlast = 1;
    s.status = ST_SUCCESS;

    c.load_y(V_Z0);
    if (!(tout > t0)) { c.store_y(V_Z0); return; }
    c.rhs(V_Z0, V_F);
    s.nfe++;
    if (!c.all_finite(V_F) || !c.all_finite(V_Z0)) {
        s.status = ST_NONFINITE;
        c.store_y(V_Z0);
        return;
    }
    c.set_weights(V_Z0, ctl.rtol);

    // ---- starting step (Hairer, Norsett & Wanner, order 1) ----
    double h;
    {
        const double span = tout - t0;
        const double d0 = c.wrms2(V_Z0), d1 = c.wrms2(V_F);   // squared
        double h0 = (d0 < 1e-10 || d1 < 1e-10) ? 1e-6 * span : 0.01 * sqrt(d0 * rcp(d1));
        if (h0 > span) h0 = span;
        c.axpby(V_Y, 1.0, V_Z0, h0, V_F);
        c.rhs(V_Y, V_DEL);
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

    double t = t0;
    int q = 1, qwait = 2, have_M = 0, force_setup = 1, nst_lastsetup = 0, have_ks = 0;
    double hist[QMAX + 1];
#pragma unroll
    for (int i = 0; i <= QMAX; ++i) hist[i] = 0.0;
    double gamma_M = 0.0, etamax = ETA_MAX_FIRST, h_ks = 0.0;
    int nsame = 0;    // leading entries of hist equal to the current h

    while (t < tout) {
        if (s.nst >= ctl.max_steps) { s.status = ST_TOO_MUCH_WORK; break; }
        int last = 0;
        if (t + h >= tout || tout - (t + h) <= 4.0 * 2.220446049250313e-16 * fabs(tout)) {
            const double hn = tout - t;
            c.rescale(q, hn * rcp(h));
            h = hn;
            last = 1;
            nsame = 0;
        }
        c.set_weights(V_Z0, ctl.rtol);          // Eq. wrms: weights from y^{n-1}
        int ncf = 0, nef = 0;
        double dsm2 = 0.0, l[QMAX + 1], xi[QMAX + 1], inv[QMAX + 1], Cq = 0.0;
        double gamma_acc = 0.0, il1_acc = 0.0;     // of the attempt that is accepted
        for (;;) {   // attempts
            c.predict(q);
            double il1;
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
                il1 = rcp(l[1]);
                Cq = rcp(1.0 + l[1] * xi[q]);
            }
            const double gamma = h * il1;
            gamma_acc = gamma;
            il1_acc = il1;
            const double Cq2 = Cq * Cq;
            int fresh = 0, conv = 0, fcur = 0;   // fcur: V_F holds f(z0) already
            if (force_setup || !have_M || s.nst >= nst_lastsetup + MSBP ||
                fabs(gamma * rcp(gamma_M) - 1.0) > DGMAX) {
                have_M = c.rhs_setup(V_Z0, V_F, gamma);
                s.nje++; s.nfe++;
                gamma_M = gamma; nst_lastsetup = s.nst; fresh = 1; force_setup = 0; fcur = 1;
            }
            for (;;) {   // Newton
                conv = 0;
                if (!have_M) break;
                c.newton_init();
                double delp2 = 0.0, R2 = 1.0;
                const double cstale = (gamma != gamma_M) ? 2.0 * rcp(1.0 + gamma * rcp(gamma_M)) : 1.0;
                for (int m = 0;; ++m) {
                    if (!fcur) { c.rhs(V_Y, V_F); s.nfe++; }
                    fcur = 0;
                    s.nni++;
                    c.newton_residual(h, il1);
                    c.solve(V_DEL);
                    const double dn2 = c.newton_update(cstale);
                    if (!(dn2 <= 1.7e308)) break;             // not finite
                    if (m > 0) R2 = fmax(CRDOWN * CRDOWN * R2, dn2 * rcp(delp2));
                    if (R2 * dn2 * Cq2 < NLS_COEF * NLS_COEF) { conv = 1; break; }
                    if (m + 1 == MAXCOR || (m > 0 && dn2 > RDIV * RDIV * delp2)) break;
                    delp2 = dn2;
                }
                if (conv || fresh) break;
                have_M = c.rhs_setup(V_Z0, V_F, gamma);    // stale matrix: rebuild and retry
                s.nje++; s.nfe++;
                gamma_M = gamma; nst_lastsetup = s.nst; fresh = 1; fcur = 1;
            }
            if (!conv) {   // Newton failure
                c.unpredict(q);
                s.ncf++; ncf++;
                if (ncf >= MXNCF) { s.status = ST_CONV_FAILURE; break; }
                h *= ETA_CF;
                c.rescale(q, ETA_CF);
                force_setup = 1; etamax = 1.0; last = 0; nsame = 0;
                if (t + h == t) { s.status = ST_H_TOO_SMALL; break; }
                continue;
            }
            dsm2 = Cq2 * c.wrms2(V_ACOR);
            if (dsm2 < 1.0) break;     // accept: ||LTE|| < 1
            // error-test failure
            c.unpredict(q);
            s.nef++; nef++;
            if (nef >= MXNEF) { s.status = ST_ERR_FAILURE; break; }
            if (nef < MXNEF1) {
                double eta = eta_from(dsm2, q, BIAS_Q);
                int newq = q;
                if (q > 1) {
                    double l1m = 0.0, pm = 1.0;
                    for (int i = 0; i < q - 1; ++i) { l1m += inv[i]; pm *= xi[i]; }
                    const double f = pm * rcp(l1m);
                    const double em = eta_from(c.wrms2(q) * f * f, q - 1, BIAS_QM1);
                    if (em > eta) { eta = em; newq = q - 1; }
                }
                eta = fmin(ETA_MAX_EF, fmax(ETA_MIN_EF, eta));
                if (newq < q) {
                    double nodes[QMAX], sacc = 0.0, e[QMAX + 1];
                    const double rh = rcp(h);
                    for (int i = 0; i < QMAX; ++i) {
                        sacc += hist[i];
                        nodes[i] = sacc * rh;
                    }
                    decrease_coeffs(q, nodes, e);
                    c.order_decrease(q, e);
                    q = newq; qwait = q + 1;
                }
                h *= eta;
                c.rescale(q, eta);
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
                h *= ETA_MIN_EF;
                c.rescale(q, ETA_MIN_EF);
                qwait = 2; have_ks = 0;
            }
            etamax = 1.0; last = 0; nsame = 0;
            if (t + h == t) { s.status = ST_H_TOO_SMALL; break; }
        }
        if (s.status != ST_SUCCESS) break;

        // ---- accepted step ----
        s.nst++;
        t = last ? tout : t + h;
        c.correct(q, l);
#pragma unroll
        for (int i = QMAX; i > 0; --i) hist[i] = hist[i - 1];
        hist[0] = h;
        if (last) {
            c.rec_accept(q, q, l, 0.0, gamma_acc, il1_acc);
            break;
        }

        qwait--;
        const double l1 = l[1];
        double eta = 1.0;
        int newq = q;
        const double kfac = l1 * l[q] * Cq;     // h^{q+1} y^{(q+1)}/(q+1)! = kfac * Delta
        if (BIAS_Q * BIAS_Q * dsm2 <= eta_viable2(q)) eta = eta_from(dsm2, q, BIAS_Q);
        if (qwait == 0) {
            double em = 0.0, ep = 0.0;
            if (q > 1) {
                double l1m = 0.0, pm = 1.0;
                for (int i = 0; i < q - 1; ++i) { l1m += inv[i]; pm *= xi[i]; }
                const double f = pm * rcp(l1m);
                const double d2 = c.wrms2(q) * f * f;
                if (BIAS_QM1 * BIAS_QM1 * d2 <= eta_viable2(q - 1)) em = eta_from(d2, q - 1, BIAS_QM1);
            }
            if (q < qmax && have_ks) {
                double rq = 1.0;
                const double rr = h * rcp(h_ks);
                for (int i = 0; i <= q; ++i) rq *= rr;
                double pp = 1.0;
                for (int i = 0; i <= q; ++i) pp *= xi[i];
                const double l1p = l1 + inv[q];
                const double f = pp * rcp(l1p * (q + 2));
                const double d2 = c.wrms2_lin(kfac, V_ACOR, -rq, V_KS) * f * f;
                if (BIAS_QP1 * BIAS_QP1 * d2 <= eta_viable2(q + 1)) ep = eta_from(d2, q + 1, BIAS_QP1);
            }
            if (em > eta && em >= ep) { eta = em; newq = q - 1; }
            else if (ep > eta) { eta = ep; newq = q + 1; }
        }
        if (eta < ETA_THRESH) { eta = 1.0; newq = q; }
        else eta = fmin(eta, etamax);
        c.rec_accept(q, newq == q + 1 ? q + 1 : q, l, inv[q], gamma_acc, il1_acc);
        if (newq == q + 1) c.order_increase(q, l, inv[q]);
        else if (newq == q - 1) {
            double e[QMAX + 1];
            decrease_coeffs(q, xi, e);
            c.order_decrease(q, e);
        }
        if (newq != q || qwait == 0) { q = newq; qwait = q + 1; have_ks = 0; }
        if (qwait == 1 && q < qmax) {
            c.scale(V_KS, kfac, V_ACOR);
            h_ks = h; have_ks = 1;
        }
        if (eta != 1.0) {
            h *= eta;
            c.rescale(q, eta);
            nsame = 0;
        } else if (nsame < QMAX) {
            ++nsame;
        }
        etamax = ETA_MAX;
    }
    s.qlast = q;
    c.store_y(V_Z0);
}

}  // namespace sunb
