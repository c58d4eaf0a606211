/* CPU oracle for the batched BDF integrator: TEST INFRASTRUCTURE ONLY.
 *
 * Plain C, FP64 (the step-size factors, a heuristic, in single precision:
 * see eta_from), one cell at a time (OpenMP only distributes independent
 * cells).  Only the tests, smoke() and the benchmark's CPU-baseline leg may
 * load it; the CUDA library shares no code with it.
 *
 * The method (arXiv 2405.01713, Sec. 2): each cell's ODE y' = f(t, y; p)
 * (Eq. 1) is advanced by an adaptive-order (1..5), adaptive-step linear
 * multistep (BDF) method of the CVODE kind.  A step is accepted when the WRMS
 * norm (Eq. wrms) of its local-truncation-error estimate is below one;
 * otherwise the step is cut and, possibly, the order lowered.  The implicit
 * corrector is solved by a modified Newton iteration with the stopping test
 * of Eq. stop_newton (c_eps = 0.1, c_r = 0.3), on the matrix I - gamma J with
 * a dense Jacobian (solution approaches 2A/3A of Table 1) factored by LU with
 * partial pivoting (Sec. 4.1.6), reused across iterations and steps until
 * the iteration diverges (Sec. 3.1).
 *
 * The paper does not print the BDF internals; the readings used here are:
 *  - Nordsieck history z_j = h^j y^(j)/j!, predicted by the Pascal-triangle
 *    sums, corrected by z += l * Delta, where l are the coefficients of
 *    Lambda(x) = prod_{i=1..q} (1 + x/xi_i), xi_i = (t_n - t_{n-i})/h_n
 *    (the variable-coefficient form: the corrected polynomial interpolates
 *    y_n and the q previous solution values);
 *  - local error estimate E = Delta / (1 + l_1 xi_{q+1}), exact for a
 *    solution that is a polynomial of degree q+1 when f does not depend on y;
 *  - Newton tolerance: R ||delta|| < 0.1 / C_q with C_q = 1/(1 + l_1 xi_{q+1})
 *    (the correction may use a tenth of the error-test budget); at most 3
 *    iterations, divergence when ||delta_m|| > 2 ||delta_{m-1}||; R starts
 *    at 1 in every Newton solve (it estimates the rate of the current
 *    iteration; carrying it over from earlier steps let unconverged first
 *    corrections pass the test and pollute the error estimate);
 *  - matrix rebuild (fresh J, M = I - gamma J, LU) when 20 steps have passed
 *    since the last one, when |gamma/gamma_M - 1| > 0.3, or after a Newton
 *    failure; a stale matrix scales each correction by 2/(1 + gamma/gamma_M);
 *  - step factors eta_p = 1/((b_p ||E_p||)^(1/(p+1)) + 1e-6), in single
 *    precision, with biases 6 (q-1), 6 (q), 10 (q+1); no change below 1.5; growth capped at 1e4 on
 *    the first step and 10 afterwards, and at 1 right after a failed attempt;
 *    order changes considered after q+1 steps at the current order;
 *  - error-test failure: eta in [0.1, 0.9], lower order when that allows a
 *    larger step; from the third failure of a step, eta = 0.1 at order 1,
 *    reached by lowering the order of the interpolating polynomial (its
 *    slope then comes from accepted states, not from f at a state that may
 *    sit slightly off a stiff slow manifold); seven failures end the cell
 *    (ERR_FAILURE); Newton failure: eta = 0.25, ten per step end the cell
 *    (CONV_FAILURE);
 *  - first step from the starting-step algorithm of Hairer, Norsett and
 *    Wanner (Solving ODEs I, Sec. II.4) with the WRMS norm;
 *  - every call is a cold start at order 1 and lands exactly on tout.
 *
 * Options select the variants the paper compares: a forward-difference
 * Jacobian (approaches 3A/3B), GMRES linear solves of an inexact Newton
 * iteration (approaches 1A/1B; gmres_solve), and, instead of the BDF, an
 * explicit adaptive Runge-Kutta method (Sec. 4.1.5; erk_cell).  Each
 * carries its readings beside its code.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

#define EXPORT __attribute__((visibility("default")))
#define QMAX 5

/* ---- right-hand sides: real and complex instances -------------------- */
#define REAL double
#define FN(x) x##_r
#define RE(x) (x)
#define EXPF exp
#define LOGF log
#include "rhs_impl.h"
#undef REAL
#undef FN
#undef RE
#undef EXPF
#undef LOGF

#define REAL double complex
#define FN(x) x##_c
#define RE(x) creal(x)
#define EXPF cexp
#define LOGF clog
#include "rhs_impl.h"
#undef REAL
#undef FN
#undef RE
#undef EXPF
#undef LOGF

EXPORT void orc_rhs(const orc_problem *pb, long cell, const double *y, double *f)
{
    rhs_r(pb, cell, y, f);
}

/* Dense Jacobian J[i*n + j] = d f_i / d y_j.
 * mode 0: complex step, J e_j = Im f(y + i s e_j) / s with s = 1e-30 (no
 * subtractive cancellation, so exact to rounding);
 * mode 1: forward difference quotient (the numerical Jacobian of solution
 * approaches 3A/3B, Table 1) with increment max(sqrt(eps)|y_j|, sqrt(eps)/w_j). */
EXPORT void orc_jac(const orc_problem *pb, long cell, const double *y,
                    const double *f0, const double *w, int mode, double *J)
{
    const int n = pb->n;
    if (mode == 0) {
        double complex yc[n], fc[n];
        const double s = 1e-30;
        for (int j = 0; j < n; ++j) {
            for (int k = 0; k < n; ++k) yc[k] = y[k];
            yc[j] = y[j] + I * s;
            rhs_c(pb, cell, yc, fc);
            for (int i = 0; i < n; ++i) J[i * n + j] = cimag(fc[i]) / s;
        }
    } else {
        double yp[n], fp[n];
        const double se = sqrt(DBL_EPSILON);
        for (int j = 0; j < n; ++j) {
            memcpy(yp, y, sizeof(double) * n);
            double inc = fmax(se * fabs(y[j]), se / w[j]);
            yp[j] = y[j] + inc;
            inc = yp[j] - y[j];
            rhs_r(pb, cell, yp, fp);
            for (int i = 0; i < n; ++i) J[i * n + j] = (fp[i] - f0[i]) / inc;
        }
    }
}

/* ---- dense LU with partial pivoting (Sec. 4.1.6, "dense direct") ----------
 * Row pivoting, pivot = the first row of largest magnitude in the column.
 * piv[k] is the row exchanged with row k at elimination step k.  Returns 0,
 * or k+1 when column k has no nonzero pivot. */
EXPORT int orc_lu_factor(int n, double *A, int32_t *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double amax = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > amax) { amax = fabs(A[i * n + k]); p = i; }
        piv[k] = p;
        if (amax == 0.0) return k + 1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        for (int i = k + 1; i < n; ++i) {
            double lik = A[i * n + k] / A[k * n + k];
            A[i * n + k] = lik;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= lik * A[k * n + j];
        }
    }
    return 0;
}

EXPORT void orc_lu_solve(int n, const double *LU, const int32_t *piv, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int i = 1; i < n; ++i)
        for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

/* ---- BDF coefficient algebra ------------------------------------------ */

/* xi[i-1] = xi_i = (t_n - t_{n-i}) / h for i = 1..m, from the current step h
 * and the previous accepted step sizes hist[0] = h_{n-1}, hist[1] = h_{n-2}..
 * (zero where the history does not reach: a repeated node, i.e. the Taylor
 * start). */
static void bdf_xi(int m, double h, const double *hist, double *xi)
{
    double s = h;
    xi[0] = 1.0;
    for (int i = 1; i < m; ++i) { s += hist[i - 1]; xi[i] = s / h; }
}

/* l[0..q]: coefficients of Lambda(x) = prod_{i=1..q} (1 + x/xi_i). */
/* Typical-value absolute tolerances (Sec. 4.1.3, Eq. eta): for each
 * component i of the C cells y [C x n] (row-major), the typical value is
 *   ytilde_i = (min_c y_ci + max_c y_ci) / 2
 * over the whole batch, and atol_i = eta * ytilde_i.  Where the typical
 * value is not a positive finite number (a component that is zero or
 * negative everywhere, or NaN in some cell), it takes the paper's default
 * ytilde_i = 1.  Evaluated as eta * (0.5 * (min + max)). */
EXPORT void orc_typical_atol(const double *y, long C, int n, double eta, double *atol)
{
    for (int i = 0; i < n; ++i) {
        double mn = 0.0, mx = 0.0;
        int nan = 0;
        for (long c = 0; c < C; ++c) {
            const double v = y[c * n + i];
            if (v != v) { nan = 1; continue; }
            if (c == 0 || v < mn) mn = v;
            if (c == 0 || v > mx) mx = v;
        }
        double yt = 0.5 * (mn + mx);
        if (nan || C < 1 || !(yt > 0.0) || !(yt <= 1.7976931348623157e308)) yt = 1.0;
        atol[i] = eta * yt;
    }
}

EXPORT void orc_bdf_l(int q, const double *xi, double *l)
{
    l[0] = 1.0;
    for (int j = 1; j <= q; ++j) l[j] = 0.0;
    for (int i = 0; i < q; ++i)
        for (int j = i + 1; j >= 1; --j) l[j] += l[j - 1] / xi[i];
}

/* C_q = 1 / (1 + l_1 xi_{q+1}): the estimate E = C_q Delta.  The
 * integrator and the fixed-step routine call this same function. */
static double error_constant(double l1, double xi_qp1)
{
    return 1.0 / (1.0 + l1 * xi_qp1);
}

EXPORT double orc_error_constant(int q, const double *xi)
{
    double l[QMAX + 2];
    orc_bdf_l(q, xi, l);
    return error_constant(l[1], xi[q]);
}

/* Nordsieck prediction z <- z Pascal(q): the repeated in-place sums
 * z_{j-1} += z_j (the integrator and the fixed-step routine). */
static void predict(int q, int n, double *z)
{
    for (int k = 0; k < q; ++k)
        for (int j = q; j > k; --j)
            for (int i = 0; i < n; ++i) z[(j - 1) * n + i] += z[j * n + i];
}

/* Lower the order of the Nordsieck array z (columns 0..q, n values each) by
 * one, keeping the polynomial's values at x = 0 and x = -nodes[i],
 * i < q-1: subtract z_q * x * prod_{i<q-1} (x + nodes[i]). */
EXPORT void orc_order_decrease(int q, int n, double *z, const double *nodes)
{
    double e[QMAX + 1] = {1.0, 0, 0, 0, 0, 0};
    for (int i = 0; i < q - 1; ++i) {
        for (int j = i + 1; j >= 1; --j) e[j] = e[j - 1] + e[j] * nodes[i];
        e[0] *= nodes[i];
    }
    for (int j = 1; j < q; ++j)
        for (int k = 0; k < n; ++k) z[j * n + k] -= e[j - 1] * z[q * n + k];
    for (int k = 0; k < n; ++k) z[q * n + k] = 0.0;
}

/* Raise the order by one after a step at order q with correction acor and
 * corrector coefficients l: add acor * (x/xi_{q+1}) * Lambda(x), the degree
 * q+1 term that makes the polynomial also interpolate y_{n-q-1}. */
EXPORT void orc_order_increase(int q, int n, double *z, const double *acor,
                               const double *l, double xi_qp1)
{
    for (int k = 0; k < n; ++k) z[(q + 1) * n + k] = 0.0;
    for (int j = 1; j <= q + 1; ++j)
        for (int k = 0; k < n; ++k) z[j * n + k] += acor[k] * l[j - 1] / xi_qp1;
}

/* ---- vector helpers ---------------------------------------------------- */
static double wrms(int n, const double *v, const double *w)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) { double t = v[i] * w[i]; s += t * t; }
    return sqrt(s / n);
}

static void set_weights(int n, const double *y, double rtol, const double *atol, double *w)
{
    for (int i = 0; i < n; ++i) w[i] = 1.0 / (rtol * fabs(y[i]) + atol[i]);
}

static int all_finite(int n, const double *v)
{
    for (int i = 0; i < n; ++i) if (!isfinite(v[i])) return 0;
    return 1;
}

static void rescale(int q, int n, double *z, double eta)
{
    double f = 1.0;
    for (int j = 1; j <= q; ++j) {
        f *= eta;
        for (int k = 0; k < n; ++k) z[j * n + k] *= f;
    }
}

/* Step factor eta_p = 1/((b ||E_p||)^(1/(p+1)) + 1e-6), in single
 * precision: L = log2(b ||E_p||) rounded to float, r = 2^(L/(p+1)) and
 * eta = 1/(r + 1e-6) in float.  The paper fixes no precision for this
 * heuristic, which only scales h; the CUDA path computes it in single
 * precision, and the decisions it makes (keep h below 1.5, the order of the
 * largest factor) are taken here in the same precision.  ||E|| = 0 gives
 * L = -inf and eta = 1e6 (above every growth cap). */
static double eta_from(double dsm, int p, double bias)
{
    const float L = (float)log2(bias * dsm);
    const float r = exp2f(L / (float)(p + 1));
    return (double)(1.0f / (r + 1e-6f));
}

/* Step factor and order after an accepted step at order q (Sec. 2: the
 * next step size, and the order, are selected from the error estimates).
 * Readings: eta_p = 1/((b_p ||E_p||)^(1/(p+1)) + 1e-6) with biases 6 for
 * q-1 and q and 10 for q+1; the orders q-1 and q+1 are considered only
 * when qwait == 0 (q+1 steps taken at q); ||E_{q-1}|| from the corrected
 * z_q, ||E_{q+1}|| from the change of the scaled (q+1)th derivative since
 * the saved correction ksave of step size h_ksave; no change below
 * eta = 1.5; growth capped at etamax.  z is the corrected array, acor the
 * correction Delta, dsm = C_q ||Delta||; tmp2 is scratch [n].  Returns eta,
 * the order in *newq. */
static double choose_step(int n, int q, int qmax, int qwait, const double *z, const double *acor,
                          const double *w, const double *xi, const double *l, double dsm,
                          int have_ksave, const double *ksave, double h, double h_ksave,
                          double etamax, double *tmp2, int *newq_out)
{
    const double l1 = l[1];
    double eta = eta_from(dsm, q, 6.0);
    int newq = q;
    const double kfac = l1 * l[q] / (1.0 + l1 * xi[q]);
    if (qwait == 0) {
        double em = 0.0, ep = 0.0;
        if (q > 1) {
            double l1m = 0.0, pm = 1.0;
            for (int i = 0; i < q - 1; ++i) { l1m += 1.0 / xi[i]; pm *= xi[i]; }
            em = eta_from(wrms(n, z + q * n, w) * pm / l1m, q - 1, 6.0);
        }
        if (q < qmax && have_ksave) {
            double rq = pow(h / h_ksave, q + 1), pp = 1.0, l1p = l1 + 1.0 / xi[q];
            for (int i = 0; i <= q; ++i) pp *= xi[i];
            for (int i = 0; i < n; ++i) tmp2[i] = (kfac * acor[i] - rq * ksave[i]) / (q + 2);
            ep = eta_from(wrms(n, tmp2, w) * pp / l1p, q + 1, 10.0);
        }
        if (em > eta && em >= ep) { eta = em; newq = q - 1; }
        else if (ep > eta) { eta = ep; newq = q + 1; }
    }
    if (eta < 1.5) { eta = 1.0; newq = q; }
    else eta = fmin(eta, etamax);
    *newq_out = newq;
    return eta;
}

/* The linear solve of the inexact Newton iteration (solution approaches
 * 1A/1B of Table 1; Eqs. linear and stop_linear, Sec. 2): GMRES on the
 * system scaled by S = diag(w) and unpreconditioned,
 *   (S M S^-1) xt = S b,  x = S^-1 xt,  M v = v - gamma J v,
 * with J v by a forward difference along v at the current iterate y,
 *   J v = (f(y + sig v) - f(y)) / sig,  sig = 1 / ||v||_wrms.
 * Modified Gram-Schmidt, Givens rotations; the residual norm is |g_{k+1}|
 * from the rotations.  Stops when it is at most tol (the 2-norm of the
 * scaled residual) or after maxl = min(n, GMRES_MAXL) iterations (no
 * restarts: the Krylov space may grow to the whole system), returning the
 * approximation so far (x = 0 when ||S b|| <= tol).  b is overwritten by x.
 * Counts its f evaluations in *nfe; returns the iterations taken. */
#define GMRES_MAXL 64
static int gmres_solve(const orc_problem *pb, long cell, const double *y, const double *fy,
                       const double *w, double gamma, double tol, double *b, int32_t *nfe)
{
    const int n = pb->n, maxl = n < GMRES_MAXL ? n : GMRES_MAXL;
    double V[(maxl + 1) * n], H[(maxl + 1) * maxl], cs[maxl], sn[maxl];
    double g[maxl + 1], c[maxl], u[n], yt[n], ft[n];
    double beta = 0.0;
    for (int i = 0; i < n; ++i) { V[i] = w[i] * b[i]; beta += V[i] * V[i]; }
    beta = sqrt(beta);
    for (int i = 0; i < n; ++i) b[i] = 0.0;
    if (!(beta > tol)) return 0;
    for (int i = 0; i < n; ++i) V[i] /= beta;
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < maxl; ++j) {
        double *vj = V + j * n, *vn = V + (j + 1) * n;
        /* S M S^-1 v_j */
        double nu2 = 0.0;
        for (int i = 0; i < n; ++i) { u[i] = vj[i] / w[i]; nu2 += (u[i] * w[i]) * (u[i] * w[i]); }
        const double sig = 1.0 / sqrt(nu2 / n);
        for (int i = 0; i < n; ++i) yt[i] = y[i] + sig * u[i];
        rhs_r(pb, cell, yt, ft);
        (*nfe)++;
        for (int i = 0; i < n; ++i) vn[i] = w[i] * (u[i] - gamma * ((ft[i] - fy[i]) / sig));
        /* modified Gram-Schmidt */
        for (int m = 0; m <= j; ++m) {
            double h = 0.0;
            for (int i = 0; i < n; ++i) h += vn[i] * V[m * n + i];
            H[m * maxl + j] = h;
            for (int i = 0; i < n; ++i) vn[i] -= h * V[m * n + i];
        }
        double hn = 0.0;
        for (int i = 0; i < n; ++i) hn += vn[i] * vn[i];
        hn = sqrt(hn);
        H[(j + 1) * maxl + j] = hn;
        /* previous rotations on column j, then the one that zeroes H[j+1][j] */
        for (int m = 0; m < j; ++m) {
            const double a = H[m * maxl + j], bb = H[(m + 1) * maxl + j];
            H[m * maxl + j] = cs[m] * a + sn[m] * bb;
            H[(m + 1) * maxl + j] = -sn[m] * a + cs[m] * bb;
        }
        const double a = H[j * maxl + j], bb = hn, r = sqrt(a * a + bb * bb);
        cs[j] = r > 0.0 ? a / r : 1.0;
        sn[j] = r > 0.0 ? bb / r : 0.0;
        H[j * maxl + j] = r;
        H[(j + 1) * maxl + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        if (fabs(g[j + 1]) <= tol || !(hn > 0.0)) break;
        for (int i = 0; i < n; ++i) vn[i] /= hn;
    }
    /* H(0:k, 0:k) c = g(0:k), x = S^-1 sum_m c_m v_m */
    for (int i = k - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int m = i + 1; m < k; ++m) sacc -= H[i * maxl + m] * c[m];
        c[i] = sacc / H[i * maxl + i];
    }
    for (int i = 0; i < n; ++i) {
        double xt = 0.0;
        for (int m = 0; m < k; ++m) xt += c[m] * V[m * n + i];
        b[i] = xt / w[i];
    }
    return k;
}

/* gmres_solve for tests: x into b, the iterations and f evaluations returned. */
EXPORT int orc_gmres(const orc_problem *pb, long cell, const double *y, const double *w, double gamma,
                     double tol, double *b, int32_t *nfe)
{
    double fy[pb->n];
    rhs_r(pb, cell, y, fy);
    return gmres_solve(pb, cell, y, fy, w, gamma, tol, b, nfe);
}

/* One modified Newton solve of the corrector equation (Sec. 2):
 *   G(y) = y - gamma f(t_n, y) - a_n = 0,  a_n = z0 - z1/l_1,
 * from the prediction y = z0, written for the correction acor = y - z0 as
 * delta = M^-1 ((h f(y) - z1)/l_1 - acor) with the factors of
 * M = I - gamma_M J (or GMRES for the inexact iteration); a stale matrix
 * (gamma != gamma_M) scales each correction by 2/(1 + gamma/gamma_M).
 * Stopping test of Eq. stop_newton: after correction m,
 *   R = max(c_r R, ||delta_m|| / ||delta_{m-1}||)  (c_r = 0.3, R = 1 at m = 0)
 *   converged when R ||delta_m|| < c_eps eps = 0.1 / C_q  (WRMS norms);
 * at most 3 corrections; divergence when ||delta_m|| > 2 ||delta_{m-1}||.
 * Returns 1 on convergence; acor and ycur hold the last iterate, f and del
 * the last f and correction; nfe and nni count f evaluations and
 * iterations; *iters (nullable) receives the number of corrections. */
static int newton_solve(const orc_problem *pb, long cell, const double *z, double h, double l1,
                        double gamma, double gamma_M, double Cq, const double *M, const int32_t *piv,
                        int krylov, const double *w, double *acor, double *ycur, double *f, double *del,
                        int32_t *nfe, int32_t *nni, int *iters)
{
    const int n = pb->n;
    int conv = 0, m;
    for (int i = 0; i < n; ++i) { acor[i] = 0.0; ycur[i] = z[i]; }
    double delp = 0.0, R = 1.0;
    for (m = 0;; ++m) {
        rhs_r(pb, cell, ycur, f);
        (*nfe)++; (*nni)++;
        for (int i = 0; i < n; ++i) del[i] = (h * f[i] - z[n + i]) / l1 - acor[i];
        if (krylov) {
            /* Eq. stop_linear: c_l = 0.05 of the Newton tolerance 0.1/C_q,
             * a WRMS bound, i.e. sqrt(n) times it in the scaled 2-norm */
            gmres_solve(pb, cell, ycur, f, w, gamma, 0.05 * (0.1 / Cq) * sqrt((double)n), del, nfe);
        } else {
            orc_lu_solve(n, M, piv, del);
        }
        if (gamma != gamma_M) {
            double c = 2.0 / (1.0 + gamma / gamma_M);
            for (int i = 0; i < n; ++i) del[i] *= c;
        }
        for (int i = 0; i < n; ++i) { acor[i] += del[i]; ycur[i] = z[i] + acor[i]; }
        double dn = wrms(n, del, w);
        if (!isfinite(dn)) break;
        if (m > 0) R = fmax(0.3 * R, dn / delp);
        if (R * dn * Cq < 0.1) { conv = 1; break; }  /* Eq. stop_newton */
        if (m + 1 == 3 || (m > 0 && dn > 2.0 * delp)) break;
        delp = dn;
    }
    if (iters) *iters = m + 1;
    return conv;
}

/* newton_solve for tests, with given factors of M (LU only): z [2, n]
 * (prediction z0 and z1), weights w; acor and y receive the last iterate,
 * *iters the number of corrections; returns 1 on convergence. */
EXPORT int orc_newton_solve(const orc_problem *pb, long cell, const double *z, double h, double l1,
                            double gamma, double gamma_M, double Cq, const double *M,
                            const int32_t *piv, const double *w, double *acor, double *y, int *iters)
{
    const int n = pb->n;
    double f[n], del[n];
    int32_t nfe = 0, nni = 0;
    return newton_solve(pb, cell, z, h, l1, gamma, gamma_M, Cq, M, piv, 0, w, acor, y, f, del,
                        &nfe, &nni, iters);
}

/* Matrix set-up: J at (t, y), M = I - gamma J, LU. Returns 0 on success. */
static int setup_matrix(const orc_problem *pb, long cell, const double *y,
                        const double *w, int jac_mode, double gamma,
                        double *M, int32_t *piv, double *ftmp)
{
    const int n = pb->n;
    if (jac_mode == 1) rhs_r(pb, cell, y, ftmp);
    orc_jac(pb, cell, y, ftmp, w, jac_mode, M);
    for (int i = 0; i < n * n; ++i) M[i] = -gamma * M[i];
    for (int i = 0; i < n; ++i) M[i * n + i] += 1.0;
    if (!all_finite(n * n, M)) return -1;
    return orc_lu_factor(n, M, piv) ? -1 : 0;
}

/* Starting step of Hairer, Norsett & Wanner (Solving ODEs I, II.4), order 1,
 * with the WRMS norm of Eq. wrms; bounded by the interval length. */
static double initial_step(const orc_problem *pb, long cell, double t0, double tout,
                           const double *y0, const double *f0, const double *w,
                           double *ytmp, double *ftmp, int *nfe)
{
    const int n = pb->n;
    const double span = tout - t0;
    double d0 = wrms(n, y0, w), d1 = wrms(n, f0, w);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 * span : 0.01 * d0 / d1;
    if (h0 > span) h0 = span;
    for (int i = 0; i < n; ++i) ytmp[i] = y0[i] + h0 * f0[i];
    rhs_r(pb, cell, ytmp, ftmp);
    ++*nfe;
    for (int i = 0; i < n; ++i) ytmp[i] = (ftmp[i] - f0[i]) / h0;
    double d2 = wrms(n, ytmp, w);
    double dm = fmax(d1, d2);
    double h1 = (dm <= 1e-15) ? fmax(1e-6 * span, h0 * 1e-3) : sqrt(0.01 / dm);
    double h = fmin(100.0 * h0, h1);
    if (!(h > 0.0)) h = 1e-6 * span;
    return fmin(h, span);
}

/* ---- discrete-adjoint tape --------------------------------------------
 * The forward map of one cell, frozen: the initial array [y0, h0 f(y0)],
 * then per accepted step n
 *   Z_pre  = P_n Z_{n-1}      (column map: rescales and order decreases
 *                              applied since the previous accepted step)
 *   Z_pred = Z_pre . Pascal   (prediction)
 *   y_n    : y - gamma f(y) - (z0_pred - z1_pred / l_1) = 0
 *   Z_n    = Z_pred + c_n (y_n - z0_pred)   (c = l, plus the terms of an
 *                              order increase decided after the step)
 * Record layout (doubles): y_n [n], P [6][6] (row = output column,
 * column = input column), c [6], gamma, 1/l_1, q, q_out (highest column of
 * Z_n), then the control decisions of the step: h_n and the numbers of
 * Newton and error-test failures of its rejected attempts.  Step sizes and
 * orders are frozen; each corrector counts as solved exactly (implicit
 * function theorem with the exact Jacobian).  have_states: the records'
 * y_n are states of a forward run (0 for a map built from decisions alone,
 * whose replay starts each Newton solve from the prediction). */
#define TAPE_R(n) ((n) + 49)
typedef struct {
    int n, cap, count, overflow, have_states;
    double h0;
    double *y0;     /* [n] */
    double *rec;    /* [cap][TAPE_R(n)] */
    double P[36];   /* map accumulated since the last accepted step */
} orc_tape;

static void tape_reset_map(orc_tape *tp)
{
    for (int i = 0; i < 36; ++i) tp->P[i] = (i % 7 == 0) ? 1.0 : 0.0;
}

/* the column operations of the integrator, mirrored on the tape's map */
static void tape_rescale(orc_tape *tp, int q, double eta)
{
    if (!tp) return;
    double f = 1.0;
    for (int o = 1; o <= q; ++o) {
        f *= eta;
        for (int i = 0; i < 6; ++i) tp->P[o * 6 + i] *= f;
    }
}

static void tape_decrease(orc_tape *tp, int q, const double *nodes)
{
    if (!tp) return;
    orc_order_decrease(q, 6, tp->P, nodes);   /* rows of P act as columns */
}

static void tape_record(orc_tape *tp, const double *y, const double *c, double gamma,
                        double il1, int q, int q_out, double h, int ncf, int nef)
{
    if (!tp) return;
    if (tp->count >= tp->cap) { tp->overflow = 1; return; }
    const int n = tp->n;
    double *r = tp->rec + (size_t)tp->count * TAPE_R(n);
    if (y) memcpy(r, y, sizeof(double) * n);
    else memset(r, 0, sizeof(double) * n);
    memcpy(r + n, tp->P, sizeof(double) * 36);
    memcpy(r + n + 36, c, sizeof(double) * 6);
    r[n + 42] = gamma;
    r[n + 43] = il1;
    r[n + 44] = q;
    r[n + 45] = q_out;
    r[n + 46] = h;
    r[n + 47] = ncf;
    r[n + 48] = nef;
    tp->count++;
}

/* ---- one cell, one call: t0 -> tout ------------------------------------- */
static int bdf_cell(const orc_problem *pb, long cell, double *y, double t0,
                    double tout, const orc_options *op, orc_stats *st,
                    double *hlast, orc_tape *tp)
{
    const int n = pb->n;
    const int qmax = op->max_order < 1 ? 1 : (op->max_order > QMAX ? QMAX : op->max_order);
    double *z = calloc((size_t)(QMAX + 2) * n, sizeof(double));
    double *zsave = calloc((size_t)(QMAX + 2) * n, sizeof(double));
    double *M = malloc(sizeof(double) * n * n);
    int32_t *piv = malloc(sizeof(int32_t) * n);
    double *w = malloc(sizeof(double) * n), *f = malloc(sizeof(double) * n);
    double *acor = malloc(sizeof(double) * n), *ycur = malloc(sizeof(double) * n);
    double *del = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    double *tmp2 = malloc(sizeof(double) * n), *ksave = malloc(sizeof(double) * n);

    orc_stats s = {0, 0, 0, 0, 0, 0, 1, ORC_SUCCESS};
    double t = t0, h = 0.0;
    int q = 1, qwait = 2, have_M = 0, force_setup = 1, nst_lastsetup = 0;
    int have_ksave = 0;
    double hist[QMAX + 1] = {0}, gamma_M = 0.0, etamax = 1e4, h_ksave = 0.0;

    if (!(tout > t0)) goto done_copy;
    memcpy(z, y, sizeof(double) * n);
    rhs_r(pb, cell, y, f);
    s.nfe++;
    if (!all_finite(n, f) || !all_finite(n, y)) { s.status = ORC_NONFINITE; goto done_copy; }
    set_weights(n, y, op->rtol, op->atol, w);
    h = initial_step(pb, cell, t0, tout, y, f, w, ycur, tmp, &s.nfe);
    for (int k = 0; k < n; ++k) z[n + k] = h * f[k];
    if (tp) {
        memcpy(tp->y0, y, sizeof(double) * n);
        tp->h0 = h;
        tape_reset_map(tp);
    }

    while (t < tout) {
        if (s.nst >= op->max_steps) { s.status = ORC_TOO_MUCH_WORK; break; }
        /* land exactly on tout: clip a step that would reach or pass it */
        int last = 0;
        if (t + h >= tout || tout - (t + h) <= 4.0 * DBL_EPSILON * fabs(tout)) {
            double hn = tout - t;
            rescale(q, n, z, hn / h);
            tape_rescale(tp, q, hn / h);
            h = hn;
            last = 1;
        }
        set_weights(n, z, op->rtol, op->atol, w);   /* Eq. wrms: w from y^{n-1} */
        int ncf = 0, nef = 0;
        double dsm = 0.0, Cq = 0.0, l[QMAX + 2], xi[QMAX + 2];
        for (;;) {  /* attempts */
            memcpy(zsave, z, sizeof(double) * (q + 1) * n);
            predict(q, n, z);
            bdf_xi(q + 1, h, hist, xi);
            orc_bdf_l(q, xi, l);
            const double l1 = l[1], gamma = h / l1;
            Cq = error_constant(l1, xi[q]);
            int fresh = 0, conv = 0;
            const int krylov = op->lin_solver == 1;
            if (krylov) { have_M = 1; fresh = 1; gamma_M = gamma; }   /* no matrix to keep */
            else if (force_setup || !have_M || s.nst >= nst_lastsetup + 20 ||
                fabs(gamma / gamma_M - 1.0) > 0.3) {
                have_M = setup_matrix(pb, cell, z, w, op->jac_mode, gamma, M, piv, tmp) == 0;
                s.nje++;
                gamma_M = gamma; nst_lastsetup = s.nst; fresh = 1; force_setup = 0;
            }
            for (;;) {  /* Newton on G(y) = y - gamma f(tn, y) - a_n, a_n = z0 - z1/l1 */
                conv = 0;
                if (!have_M) break;
                conv = newton_solve(pb, cell, z, h, l1, gamma, gamma_M, Cq, M, piv, krylov, w,
                                    acor, ycur, f, del, &s.nfe, &s.nni, NULL);
                if (conv || fresh) break;
                /* stale matrix: rebuild at the predicted state and retry */
                have_M = setup_matrix(pb, cell, z, w, op->jac_mode, gamma, M, piv, tmp) == 0;
                s.nje++;
                gamma_M = gamma; nst_lastsetup = s.nst; fresh = 1;
            }
            if (!conv) {  /* Newton failure */
                memcpy(z, zsave, sizeof(double) * (q + 1) * n);
                s.ncf++; ncf++;
                if (ncf >= 10) { s.status = ORC_CONV_FAILURE; break; }
                h *= 0.25; rescale(q, n, z, 0.25); tape_rescale(tp, q, 0.25);
                force_setup = 1; etamax = 1.0; last = 0;
                if (t + h == t) { s.status = ORC_H_TOO_SMALL; break; }
                continue;
            }
            dsm = Cq * wrms(n, acor, w);
            if (dsm < 1.0) break;   /* accept: ||LTE|| < 1 (Eq. wrms) */
            /* error-test failure */
            memcpy(z, zsave, sizeof(double) * (q + 1) * n);
            s.nef++; nef++;
            if (nef >= 7) { s.status = ORC_ERR_FAILURE; break; }
            double eta;
            if (nef < 3) {
                eta = eta_from(dsm, q, 6.0);
                int newq = q;
                if (q > 1) {
                    double l1m = 0.0, pm = 1.0;
                    for (int i = 0; i < q - 1; ++i) { l1m += 1.0 / xi[i]; pm *= xi[i]; }
                    double em = eta_from(wrms(n, z + q * n, w) * pm / l1m, q - 1, 6.0);
                    if (em > eta) { eta = em; newq = q - 1; }
                }
                eta = fmin(0.9, fmax(0.1, eta));
                if (newq < q) {
                    double nodes[QMAX], sacc = 0.0;
                    for (int i = 0; i < q - 1; ++i) { sacc += hist[i]; nodes[i] = sacc / h; }
                    orc_order_decrease(q, n, z, nodes);
                    tape_decrease(tp, q, nodes);
                    q = newq; qwait = q + 1;
                }
                h *= eta; rescale(q, n, z, eta); tape_rescale(tp, q, eta);
            } else {
                /* from the third failure: order 1 and eta = 0.1; the order
                 * is lowered through the interpolating polynomials, which
                 * keeps the line through the last two accepted states */
                eta = 0.1;
                if (q > 1) {
                    double nodes[QMAX], sacc = 0.0;
                    for (int i = 0; i < q - 1; ++i) { sacc += hist[i]; nodes[i] = sacc / h; }
                    for (; q > 1; --q) { orc_order_decrease(q, n, z, nodes); tape_decrease(tp, q, nodes); }
                }
                h *= eta; rescale(q, n, z, eta); tape_rescale(tp, q, eta);
                qwait = 2; have_ksave = 0;
            }
            etamax = 1.0; last = 0;
            if (t + h == t) { s.status = ORC_H_TOO_SMALL; break; }
        }
        if (s.status != ORC_SUCCESS) break;

        /* accepted step */
        s.nst++;
        t = last ? tout : t + h;
        for (int j = 0; j <= q; ++j)
            for (int i = 0; i < n; ++i) z[j * n + i] += l[j] * acor[i];
        for (int i = QMAX; i > 0; --i) hist[i] = hist[i - 1];
        hist[0] = h;
        double cvec[6] = {0, 0, 0, 0, 0, 0};
        for (int j = 0; j <= q; ++j) cvec[j] = l[j];
        if (last) {
            tape_record(tp, z, cvec, h / l[1], 1.0 / l[1], q, q, h, ncf, nef);
            break;
        }

        /* step size and order for the next step */
        qwait--;
        int newq;
        /* scaled (q+1)-th derivative estimate h^{q+1} y^{(q+1)}/(q+1)! */
        const double kfac = l[1] * l[q] / (1.0 + l[1] * xi[q]);
        double eta = choose_step(n, q, qmax, qwait, z, acor, w, xi, l, dsm, have_ksave, ksave, h, h_ksave,
                                 etamax, tmp2, &newq);
        if (newq == q + 1)
            for (int j = 1; j <= q + 1; ++j) cvec[j] += l[j - 1] / xi[q];
        tape_record(tp, z, cvec, h / l[1], 1.0 / l[1], q, newq == q + 1 ? q + 1 : q, h, ncf, nef);
        if (tp) tape_reset_map(tp);
        if (newq == q + 1) orc_order_increase(q, n, z, acor, l, xi[q]);
        else if (newq == q - 1) { orc_order_decrease(q, n, z, xi); tape_decrease(tp, q, xi); }
        if (newq != q || qwait == 0) { q = newq; qwait = q + 1; have_ksave = 0; }
        if (qwait == 1 && q < qmax) {
            for (int i = 0; i < n; ++i) ksave[i] = kfac * acor[i];
            h_ksave = h; have_ksave = 1;
        }
        h *= eta;
        rescale(q, n, z, eta);
        tape_rescale(tp, q, eta);
        etamax = 10.0;
    }
    memcpy(y, z, sizeof(double) * n);
    s.qlast = q;
    goto done;
done_copy:
    s.qlast = q;
done:
    if (st) *st = s;
    if (hlast) *hlast = h;
    free(z); free(zsave); free(M); free(piv); free(w); free(f); free(acor);
    free(ycur); free(del); free(tmp); free(tmp2); free(ksave);
    return s.status;
}

/* ---- explicit Runge-Kutta (the explicit alternative of Sec. 4.1.5) -----
 * The paper compares CVODE's implicit BDF with a fourth-order explicit,
 * adaptive-step method of ARKODE (Sec. 2: explicit RK with step adaptivity
 * from an embedded error estimate under the same WRMS test) and reports
 * about five right-hand sides per step; it does not name the table.
 * Reading: Merson's five-stage pair, order 4 with an embedded order-3
 * solution (Merson 1957; Hairer, Norsett & Wanner, Solving ODEs I, II.4),
 * advancing with the order-4 weights:
 *   k_j = f(y_n + h sum_{m<j} a_jm k_m),  y_{n+1} = y_n + h sum b_j k_j,
 *   E = h sum (b_j - bh_j) k_j,  accept iff ||E||_wrms < 1 (Eq. wrms, the
 *   weights from y_n as in the BDF),
 * step factor eta = 0.9 (1/||E||)^(1/4) (the embedded order 3, plus one),
 * at most 10 after an accepted step (1e4 after the first), at least 0.1,
 * at most 1 after a rejection and at most 0.3 from the second rejection of
 * a step on (where f is only piecewise smooth the estimate falls more
 * slowly than h^4); seven rejections of one step give ERR_FAILURE.  The starting step is the BDF's (an order-1 estimate, so the
 * first accepted steps grow it); the last step lands exactly on tout; k_1 =
 * f(y_n) is kept across a rejection.  nfe counts every f; nef the
 * rejections; qlast is 4. */
static const double ERK_A[5][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {1.0 / 3.0, 0.0, 0.0, 0.0},
    {1.0 / 6.0, 1.0 / 6.0, 0.0, 0.0},
    {1.0 / 8.0, 0.0, 3.0 / 8.0, 0.0},
    {1.0 / 2.0, 0.0, -3.0 / 2.0, 2.0},
};
static const double ERK_B[5] = {1.0 / 6.0, 0.0, 0.0, 2.0 / 3.0, 1.0 / 6.0};
static const double ERK_BH[5] = {1.0 / 10.0, 0.0, 3.0 / 10.0, 2.0 / 5.0, 1.0 / 5.0};

/* the table for tests: A [5][4], b [5], bh [5] */
EXPORT void orc_erk_table(double *A, double *b, double *bh)
{
    memcpy(A, ERK_A, sizeof(ERK_A));
    memcpy(b, ERK_B, sizeof(ERK_B));
    memcpy(bh, ERK_BH, sizeof(ERK_BH));
}

/* One step of size h from y (k1 = f(y) given): y_new and E. */
static void erk_step(const orc_problem *pb, long cell, const double *y, double h,
                     double *k /* [5][n], k[0] = f(y) */, double *ys, double *ynew, double *E)
{
    const int n = pb->n;
    for (int j = 1; j < 5; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int m = 0; m < j; ++m) s += ERK_A[j][m] * k[m * n + i];
            ys[i] = y[i] + h * s;
        }
        rhs_r(pb, cell, ys, k + j * n);
    }
    for (int i = 0; i < n; ++i) {
        double sb = 0.0, se = 0.0;
        for (int m = 0; m < 5; ++m) {
            sb += ERK_B[m] * k[m * n + i];
            se += (ERK_B[m] - ERK_BH[m]) * k[m * n + i];
        }
        ynew[i] = y[i] + h * sb;
        E[i] = h * se;
    }
}

/* Fixed step size: nsteps steps of size h from y (in place); E of the last
 * step in E_out.  Pins the order of the method and of its estimate. */
EXPORT void orc_erk_fixed(const orc_problem *pb, long cell, double h, int nsteps, double *y, double *E_out)
{
    const int n = pb->n;
    double *k = malloc(sizeof(double) * 5 * n), *ys = malloc(sizeof(double) * n);
    double *yn = malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; ++s) {
        rhs_r(pb, cell, y, k);
        erk_step(pb, cell, y, h, k, ys, yn, E_out);
        memcpy(y, yn, sizeof(double) * n);
    }
    free(k); free(ys); free(yn);
}

static int erk_cell(const orc_problem *pb, long cell, double *y, double t0, double tout,
                    const orc_options *op, orc_stats *st, double *hlast)
{
    const int n = pb->n;
    double *k = malloc(sizeof(double) * 5 * n), *ys = malloc(sizeof(double) * n);
    double *yn = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *w = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    orc_stats s = {0, 0, 0, 0, 0, 0, 4, ORC_SUCCESS};
    double t = t0, h = 0.0, etamax = 1e4;
    int nef = 0;
    if (!(tout > t0)) goto done;
    rhs_r(pb, cell, y, k);
    s.nfe++;
    if (!all_finite(n, k) || !all_finite(n, y)) { s.status = ORC_NONFINITE; goto done; }
    set_weights(n, y, op->rtol, op->atol, w);
    h = initial_step(pb, cell, t0, tout, y, k, w, ys, tmp, &s.nfe);
    int have_k1 = 1;
    while (t < tout) {
        if (s.nst >= op->max_steps) { s.status = ORC_TOO_MUCH_WORK; break; }
        int last = 0;
        if (t + h >= tout || tout - (t + h) <= 4.0 * DBL_EPSILON * fabs(tout)) { h = tout - t; last = 1; }
        set_weights(n, y, op->rtol, op->atol, w);
        if (!have_k1) { rhs_r(pb, cell, y, k); s.nfe++; have_k1 = 1; }
        erk_step(pb, cell, y, h, k, ys, yn, E);
        s.nfe += 4;
        const double err = wrms(n, E, w);
        if (err < 1.0) {          /* accept */
            memcpy(y, yn, sizeof(double) * n);
            t = last ? tout : t + h;
            s.nst++;
            have_k1 = 0;
            nef = 0;
            if (last) break;
            double eta = err > 0.0 ? 0.9 / sqrt(sqrt(err)) : etamax;
            h *= fmin(eta, etamax);
            etamax = 10.0;
            continue;
        }
        s.nef++; nef++;           /* reject (a non-finite E counts as one) */
        if (nef >= 7) { s.status = ORC_ERR_FAILURE; break; }
        double eta = isfinite(err) ? 0.9 / sqrt(sqrt(err)) : 0.1;
        if (nef >= 2) eta = fmin(eta, 0.3);
        h *= fmax(0.1, eta);
        etamax = 1.0;
        if (t + h == t) { s.status = ORC_H_TOO_SMALL; break; }
    }
done:
    if (st) *st = s;
    if (hlast) *hlast = h;
    free(k); free(ys); free(yn); free(E); free(w); free(tmp);
    return s.status;
}

/* Integrate ncells independent cells from t0 to tout (Sec. 2: one ODE
 * system per cell, all over the same outer interval dt_CFD).  y is
 * [ncells, n] (cell-contiguous "CY" order, Sec. 4.1.2).  Returns the most
 * negative per-cell status. */
EXPORT int orc_integrate(const orc_problem *pb, long ncells, double *y, double t0,
                         double tout, const orc_options *op, orc_stats *stats,
                         double *hlast, int nthreads)
{
    int worst = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) reduction(min : worst)
    for (long c = 0; c < ncells; ++c) {
        int r = op->method == 1
                    ? erk_cell(pb, c, y + (size_t)c * pb->n, t0, tout, op, stats ? stats + c : NULL,
                               hlast ? hlast + c : NULL)
                    : bdf_cell(pb, c, y + (size_t)c * pb->n, t0, tout, op,
                               stats ? stats + c : NULL, hlast ? hlast + c : NULL, NULL);
        if (r < worst) worst = r;
    }
    return worst;
}

EXPORT int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fixed step size, fixed order q: nsteps steps of size h from a given
 * Nordsieck array zinit ((q+1) x n) and step history (previous step sizes,
 * 6 entries), each corrector solved by full Newton to rounding level.
 * Returns y at the end, and for the last step the correction Delta, the
 * estimate E = C_q Delta and the corrected Nordsieck array.  Used to pin the
 * coefficients, the order and the error estimate. */
EXPORT int orc_bdf_fixed(const orc_problem *pb, long cell, int q, double h, int nsteps,
                         const double *zinit, const double *hist_init,
                         double *y_out, double *delta_out, double *est_out,
                         double *z_out)
{
    const int n = pb->n;
    double z[(QMAX + 2) * n], J[n * n], f[n], acor[n], ycur[n], del[n], w[n];
    double hist[QMAX + 1], xi[QMAX + 2], l[QMAX + 2];
    int32_t piv[n];
    memcpy(z, zinit, sizeof(double) * (q + 1) * n);
    memcpy(hist, hist_init, sizeof(double) * (QMAX + 1));
    for (int i = 0; i < n; ++i) w[i] = 1.0;
    for (int step = 0; step < nsteps; ++step) {
        predict(q, n, z);
        bdf_xi(q + 1, h, hist, xi);
        orc_bdf_l(q, xi, l);
        double gamma = h / l[1];
        for (int i = 0; i < n; ++i) { acor[i] = 0.0; ycur[i] = z[i]; }
        for (int it = 0; it < 50; ++it) {
            rhs_r(pb, cell, ycur, f);
            orc_jac(pb, cell, ycur, f, w, 0, J);
            for (int i = 0; i < n * n; ++i) J[i] = -gamma * J[i];
            for (int i = 0; i < n; ++i) J[i * n + i] += 1.0;
            if (orc_lu_factor(n, J, piv)) return -1;
            for (int i = 0; i < n; ++i) del[i] = (h * f[i] - z[n + i]) / l[1] - acor[i];
            orc_lu_solve(n, J, piv, del);
            double dmax = 0.0, ymax = 0.0;
            for (int i = 0; i < n; ++i) {
                acor[i] += del[i]; ycur[i] = z[i] + acor[i];
                dmax = fmax(dmax, fabs(del[i])); ymax = fmax(ymax, fabs(ycur[i]));
            }
            if (dmax <= 1e-15 * ymax || dmax == 0.0) break;
        }
        double Cq = error_constant(l[1], xi[q]);
        for (int j = 0; j <= q; ++j)
            for (int i = 0; i < n; ++i) z[j * n + i] += l[j] * acor[i];
        for (int i = QMAX; i > 0; --i) hist[i] = hist[i - 1];
        hist[0] = h;
        if (step == nsteps - 1) {
            for (int i = 0; i < n; ++i) {
                if (delta_out) delta_out[i] = acor[i];
                if (est_out) est_out[i] = Cq * acor[i];
            }
        }
    }
    memcpy(y_out, z, sizeof(double) * n);
    if (z_out) memcpy(z_out, z, sizeof(double) * (q + 1) * n);
    return 0;
}

/* ---- discrete adjoint (differentiation through the integrator) ---------
 * Gradient of a loss on the final state with respect to the Arrhenius
 * parameters (ln A_j, Ea_j) of the frozen forward map recorded on the tape
 * (see orc_tape).  Reverse sweep: lam is the adjoint of the Nordsieck array;
 * at each step mu = (I - gamma J(y_n))^{-T} lam_Delta, the parameter term
 * gamma (df/dtheta)^T mu is accumulated, and lam is carried back through the
 * corrector's a_n, the prediction and the column map.  J is the
 * complex-step Jacobian at y_n; df/d ln A_j is the right-hand side with the
 * rates of progress of reaction j alone (f is linear in them and
 * dq_j/d ln A_j = q_j); df/dEa_j = -df/d ln A_j / (Rc T). */
EXPORT orc_tape *orc_tape_new(int n, int cap)
{
    orc_tape *tp = calloc(1, sizeof(orc_tape));
    tp->n = n;
    tp->cap = cap;
    tp->have_states = 1;
    tp->y0 = calloc((size_t)n, sizeof(double));
    tp->rec = calloc((size_t)cap * TAPE_R(n), sizeof(double));
    tape_reset_map(tp);
    return tp;
}

EXPORT void orc_tape_free(orc_tape *tp)
{
    if (!tp) return;
    free(tp->y0);
    free(tp->rec);
    free(tp);
}

EXPORT int orc_tape_count(const orc_tape *tp) { return tp->overflow ? -1 : tp->count; }

/* Record r's column map [6][6] (row = output column), for tests. */
EXPORT int orc_tape_map(const orc_tape *tp, int r, double *P)
{
    if (r < 0 || r >= tp->count) return -1;
    memcpy(P, tp->rec + (size_t)r * TAPE_R(tp->n) + tp->n, sizeof(double) * 36);
    return 0;
}

/* The tape's contents for tests: h0 and y0 [n] into head [1 + n], the
 * records [count][n + 49] into rec (layout above); returns count. */
EXPORT int orc_tape_records(const orc_tape *tp, double *head, double *rec)
{
    head[0] = tp->h0;
    memcpy(head + 1, tp->y0, sizeof(double) * tp->n);
    memcpy(rec, tp->rec, sizeof(double) * (size_t)tp->count * TAPE_R(tp->n));
    return tp->count;
}

EXPORT int orc_forward_tape(const orc_problem *pb, long cell, double *y, double t0, double tout,
                            const orc_options *op, orc_stats *st, orc_tape *tp)
{
    tp->count = 0;
    tp->overflow = 0;
    return bdf_cell(pb, cell, y, t0, tout, op, st, NULL, tp);
}

/* F[j*n + i] = d f_i / d ln A_j at y (mechanism problems) */
EXPORT void orc_rhs_dlnA(const orc_problem *pb, long cell, const double *y, double *F)
{
    const double *prm = pb->params + (size_t)cell * pb->nparams;
    for (int j = 0; j < pb->M; ++j) rhs_mechanism_r(pb, prm, y, F + (size_t)j * pb->n, j);
}

static void theta_term(const orc_problem *pb, long cell, const double *y, const double *v,
                       double scale, double *grad, double *Fj)
{
    const int n = pb->n, M = pb->M;
    const double *prm = pb->params + (size_t)cell * pb->nparams;
    const double T = y[pb->K];
    for (int j = 0; j < M; ++j) {
        rhs_mechanism_r(pb, prm, y, Fj, j);
        double d = 0.0;
        for (int i = 0; i < n; ++i) d += Fj[i] * v[i];
        grad[2 * j] += scale * d;
        grad[2 * j + 1] += -scale * d / (ORC_RC * T);
    }
}

static int replay(const orc_problem *pb, long cell, const orc_tape *tp, double *yout, double *ys);

/* The loss is taken at the replayed final state (the map with exact
 * correctors): the forward run's states solve their correctors only to the
 * Newton tolerance, so the step history is first recomputed from the tape
 * (y0, h0 and the frozen coefficients), then swept backwards. */
EXPORT int orc_adjoint_tape(const orc_problem *pb, long cell, const orc_tape *tp,
                            const double *dLdy, double *grad)
{
    const int n = pb->n, M = pb->M, R = TAPE_R(n);
    if (tp->overflow || pb->kind != ORC_MECHANISM) return -1;
    double *ys = malloc(sizeof(double) * (size_t)n * (tp->count > 0 ? tp->count : 1));
    double *yfin = malloc(sizeof(double) * n);
    if (replay(pb, cell, tp, yfin, ys)) { free(ys); free(yfin); return -2; }
    free(yfin);
    double *lam = calloc(6 * (size_t)n, sizeof(double)), *nl = calloc(6 * (size_t)n, sizeof(double));
    double *ld = malloc(sizeof(double) * n), *J = malloc(sizeof(double) * n * n);
    double *Mt = malloc(sizeof(double) * n * n), *f = malloc(sizeof(double) * n);
    double *w = malloc(sizeof(double) * n), *Fj = malloc(sizeof(double) * n);
    int32_t *piv = malloc(sizeof(int32_t) * n);
    int rc = 0;
    for (int j = 0; j < 2 * M; ++j) grad[j] = 0.0;
    for (int i = 0; i < n; ++i) { lam[i] = dLdy[i]; w[i] = 1.0; }
    for (int r = tp->count - 1; r >= 0; --r) {
        const double *rec = tp->rec + (size_t)r * R;
        const double *y = ys + (size_t)r * n, *P = rec + n, *c = rec + n + 36;
        const double gamma = rec[n + 42], il1 = rec[n + 43];
        const int q = (int)rec[n + 44], qo = (int)rec[n + 45];
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j <= qo; ++j) s += c[j] * lam[j * n + i];
            ld[i] = s;
        }
        for (int j = q + 1; j < 6; ++j)
            for (int i = 0; i < n; ++i) lam[j * n + i] = 0.0;
        for (int i = 0; i < n; ++i) lam[i] -= ld[i];
        /* mu = (I - gamma J)^{-T} lam_Delta */
        orc_jac(pb, cell, y, f, w, 0, J);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) Mt[a * n + b] = (a == b ? 1.0 : 0.0) - gamma * J[b * n + a];
        if (orc_lu_factor(n, Mt, piv)) { rc = -2; break; }
        orc_lu_solve(n, Mt, piv, ld);      /* ld now holds mu */
        theta_term(pb, cell, y, ld, gamma, grad, Fj);
        for (int i = 0; i < n; ++i) { lam[i] += ld[i]; lam[n + i] -= il1 * ld[i]; }
        /* transpose of the prediction */
        for (int k = q - 1; k >= 0; --k)
            for (int j = k + 1; j <= q; ++j)
                for (int i = 0; i < n; ++i) lam[j * n + i] += lam[(j - 1) * n + i];
        /* transpose of the column map */
        for (int a = 0; a < 6; ++a)
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int o = 0; o < 6; ++o) s += P[o * 6 + a] * lam[o * n + i];
                nl[a * n + i] = s;
            }
        memcpy(lam, nl, sizeof(double) * 6 * n);
    }
    if (rc == 0) theta_term(pb, cell, tp->y0, lam + n, tp->h0, grad, Fj);  /* z1 = h0 f(y0) */
    free(ys);
    free(lam); free(nl); free(ld); free(J); free(Mt); free(f); free(w); free(Fj); free(piv);
    return rc;
}

/* Re-run the frozen map of the tape with the problem's current parameters,
 * each corrector solved by full Newton (fresh complex-step Jacobian every
 * iteration) to rounding level.  ys (nullable) receives the exact y_n. */
static int replay(const orc_problem *pb, long cell, const orc_tape *tp, double *yout, double *ys)
{
    const int n = pb->n, R = TAPE_R(n);
    double *Z = calloc(6 * (size_t)n, sizeof(double)), *Zp = calloc(6 * (size_t)n, sizeof(double));
    double *y = malloc(sizeof(double) * n), *f = malloc(sizeof(double) * n);
    double *J = malloc(sizeof(double) * n * n), *w = malloc(sizeof(double) * n);
    double *g = malloc(sizeof(double) * n);
    int32_t *piv = malloc(sizeof(int32_t) * n);
    int rc = 0;
    for (int i = 0; i < n; ++i) w[i] = 1.0;
    memcpy(Z, tp->y0, sizeof(double) * n);
    rhs_r(pb, cell, tp->y0, f);
    for (int i = 0; i < n; ++i) Z[n + i] = tp->h0 * f[i];
    for (int r = 0; r < tp->count && rc == 0; ++r) {
        const double *rec = tp->rec + (size_t)r * R;
        const double *P = rec + n, *c = rec + n + 36;
        const double gamma = rec[n + 42], il1 = rec[n + 43];
        const int q = (int)rec[n + 44], qo = (int)rec[n + 45];
        for (int o = 0; o < 6; ++o)
            for (int i = 0; i < n; ++i) {
                double sacc = 0.0;
                for (int a = 0; a < 6; ++a) sacc += P[o * 6 + a] * Z[a * n + i];
                Zp[o * n + i] = sacc;
            }
        for (int k = 0; k < q; ++k)
            for (int j = q; j > k; --j)
                for (int i = 0; i < n; ++i) Zp[(j - 1) * n + i] += Zp[j * n + i];
        if (tp->have_states) memcpy(y, rec, sizeof(double) * n);   /* the recorded state */
        else memcpy(y, Zp, sizeof(double) * n);                  /* the prediction */
        for (int it = 0; it < 60; ++it) {
            rhs_r(pb, cell, y, f);
            for (int i = 0; i < n; ++i) g[i] = -(y[i] - gamma * f[i] - (Zp[i] - il1 * Zp[n + i]));
            orc_jac(pb, cell, y, f, w, 0, J);
            for (int i = 0; i < n * n; ++i) J[i] = -gamma * J[i];
            for (int i = 0; i < n; ++i) J[i * n + i] += 1.0;
            if (orc_lu_factor(n, J, piv)) { rc = -2; break; }
            orc_lu_solve(n, J, piv, g);
            int done = 1;            /* converged in every component */
            for (int i = 0; i < n; ++i) {
                y[i] += g[i];
                if (fabs(g[i]) > 1e-13 * fabs(y[i]) + 1e-30) done = 0;
            }
            if (done) break;
        }
        if (ys) memcpy(ys + (size_t)r * n, y, sizeof(double) * n);
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i < n; ++i) {
                const double d = y[i] - Zp[i];
                Z[j * n + i] = (j <= qo) ? ((j <= q ? Zp[j * n + i] : 0.0) + c[j] * d) : 0.0;
            }
    }
    memcpy(yout, Z, sizeof(double) * n);
    free(Z); free(Zp); free(y); free(f); free(J); free(w); free(g); free(piv);
    return rc;
}

EXPORT int orc_replay_tape(const orc_problem *pb, long cell, const orc_tape *tp, double *yout)
{
    return replay(pb, cell, tp, yout, NULL);
}

/* replay, with the exact state of every step in ys [count, n] */
EXPORT int orc_replay_tape_states(const orc_problem *pb, long cell, const orc_tape *tp, double *yout,
                                  double *ys)
{
    return replay(pb, cell, tp, yout, ys);
}

/* ---- a step history given by its control decisions ---------------------
 * The frozen map of a cell's accepted steps rebuilt from the decisions of
 * the adaptive step and order selection alone (Sec. 2): the starting step
 * h0 and, per accepted step n, its size h_n, its order q_n, the order
 * q_out,n of the array after it (q_n + 1 after an order increase) and the
 * Newton and error-test failures of its rejected attempts.  Everything
 * else is computed here, from the oracle's own coefficient algebra:
 *  - the column map P_n: the order decreases from q_out,n-1 down to q_n,
 *    each keeping the polynomial's values at the current time and at the
 *    previous accepted times (nodes in units of h_{n-1}), then the rescale
 *    of columns 1..q_n by h_n/h_{n-1};
 *  - xi, l, gamma = h_n/l_1, 1/l_1 and the update vector c_n (l, plus the
 *    terms of an order increase, l_{j-1}/xi_{q+1}).
 * Reading: rescales and order decreases both keep one polynomial in t (a
 * rescale changes only its variable, a decrease keeps its values at the
 * current and previous accepted times), so the map does not depend on the
 * order in which an integrator applied them between two accepted steps,
 * or on the step sizes of its rejected attempts.  ys (nullable,
 * [count, n]) are states stored with the records (a forward run's, to
 * follow it); without them the replay starts each Newton solve from the
 * prediction. */
EXPORT orc_tape *orc_tape_from_decisions(int n, int count, const double *y0, double h0,
                                         const double *h, const int32_t *q, const int32_t *qo,
                                         const int32_t *ncf, const int32_t *nef, const double *ys)
{
    orc_tape *tp = orc_tape_new(n, count > 0 ? count : 1);
    memcpy(tp->y0, y0, sizeof(double) * n);
    tp->h0 = h0;
    tp->have_states = ys != NULL;
    double hist[QMAX + 1] = {0}, hprev = h0;
    int qprev = 1;                            /* [y0, h0 f(y0)] is of order 1 */
    for (int r = 0; r < count; ++r) {
        if (q[r] < 1 || q[r] > QMAX || q[r] > qprev || qo[r] < q[r] || qo[r] > q[r] + 1 ||
            !(h[r] > 0.0)) {
            orc_tape_free(tp);
            return NULL;
        }
        tape_reset_map(tp);
        if (q[r] < qprev) {
            double nodes[QMAX], sacc = 0.0;
            for (int i = 0; i < QMAX; ++i) { sacc += hist[i]; nodes[i] = sacc / hprev; }
            for (int k = qprev; k > q[r]; --k) tape_decrease(tp, k, nodes);
        }
        tape_rescale(tp, q[r], h[r] / hprev);
        double xi[QMAX + 2], l[QMAX + 2], cvec[6] = {0, 0, 0, 0, 0, 0};
        bdf_xi(q[r] + 1, h[r], hist, xi);
        orc_bdf_l(q[r], xi, l);
        for (int j = 0; j <= q[r]; ++j) cvec[j] = l[j];
        if (qo[r] == q[r] + 1)
            for (int j = 1; j <= q[r] + 1; ++j) cvec[j] += l[j - 1] / xi[q[r]];
        tape_record(tp, ys ? ys + (size_t)r * n : NULL, cvec, h[r] / l[1], 1.0 / l[1], q[r], qo[r], h[r],
                    ncf ? ncf[r] : 0, nef ? nef[r] : 0);
        for (int i = QMAX; i > 0; --i) hist[i] = hist[i - 1];
        hist[0] = h[r];
        hprev = h[r];
        qprev = qo[r];
    }
    return tp;
}

/* Corrector y - gamma f(y) - (z0 - il1 z1) = 0 solved by full Newton
 * (complex-step Jacobian every iteration) from the guess in y, to
 * |delta_i| <= 1e-13 |y_i| + 1e-30.  Returns 0, or -2 on a singular matrix. */
static int exact_corrector(const orc_problem *pb, long cell, const double *Zp, double gamma, double il1,
                           double *y)
{
    const int n = pb->n;
    double f[n], g[n], J[n * n], w1[n];
    int32_t piv[n];
    for (int i = 0; i < n; ++i) w1[i] = 1.0;
    for (int it = 0; it < 60; ++it) {
        rhs_r(pb, cell, y, f);
        for (int i = 0; i < n; ++i) g[i] = -(y[i] - gamma * f[i] - (Zp[i] - il1 * Zp[n + i]));
        orc_jac(pb, cell, y, f, w1, 0, J);
        for (int i = 0; i < n * n; ++i) J[i] = -gamma * J[i];
        for (int i = 0; i < n; ++i) J[i * n + i] += 1.0;
        if (orc_lu_factor(n, J, piv)) return -2;
        orc_lu_solve(n, J, piv, g);
        int done = 1;
        for (int i = 0; i < n; ++i) {
            y[i] += g[i];
            if (fabs(g[i]) > 1e-13 * fabs(y[i]) + 1e-30) done = 0;
        }
        if (done) break;
    }
    return 0;
}

/* Following a forward run through its recorded states and decisions (a
 * tape from orc_tape_from_decisions with ys; Sec. 2, Eq. wrms,
 * Eq. stop_newton).  The Nordsieck array is advanced with this oracle's own
 * maps, prediction and coefficients, taking the recorded y_n as each
 * step's corrector solution (Z_n = Z_pred + c_n (y_n - z0_pred)), and at
 * every step the oracle evaluates the integrator's decisions itself, with
 * weights w_i = 1/(rtol |y_{n-1,i}| + atol_i):
 *   out[0] dsm = C_q ||y_n - z0_pred||    the error test (accepted iff < 1)
 *   out[1]       C_q ||y_n - y*||         y* the exact corrector (full
 *                                          Newton): the accepted iterate's
 *                                          distance from it, in the units
 *                                          of the Newton test (0.1 there)
 *   out[2] eta, out[3] order               chosen after the step (choose_step)
 *   out[4] h_{n+1}/h_n                     recorded, where it shows that choice
 *                                          (next step not the last and
 *                                          without failures), else NaN
 *   out[5] the recorded order choice       an increase on the record, or the
 *                                          next step's order when it had no
 *                                          failures, else NaN
 *   out[6] C_q ||y* - z0_pred||           the error test of an exact corrector
 *   out[7] eta_q of that test              (the same-order step factor)
 *   out[8] 1 where orders q-1 and q+1 were considered (qwait = 0), else 0
 *   out[9] the step's rejected attempts (Newton and error-test failures)
 * out has 10 doubles per step (NaN in 2..5 for the last step, which makes
 * no choice).  The counter qwait follows the record: an increase (q_out)
 * or a choice made at qwait = 0 restarts it at the new order + 1, an order
 * decrease seen at the next step (at its accept or in a failure) restarts it
 * at that order + 1, a third error-test failure at 2.  Returns 0, or -2 if
 * an exact corrector fails. */
EXPORT int orc_follow_tape(const orc_problem *pb, long cell, const orc_tape *tp, double rtol,
                           const double *atol, int max_order, double *out)
{
    const int n = pb->n, R = TAPE_R(n), count = tp->count;
    const int qmax = max_order < 1 ? 1 : (max_order > QMAX ? QMAX : max_order);
    double *Z = calloc(6 * (size_t)n, sizeof(double)), *Zp = calloc(6 * (size_t)n, sizeof(double));
    double *w = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
    double *ystar = malloc(sizeof(double) * n), *tmp2 = malloc(sizeof(double) * n);
    double *ksave = calloc((size_t)n, sizeof(double)), *f = malloc(sizeof(double) * n);
    double *zc = calloc(6 * (size_t)n, sizeof(double));
    int rc = 0, qwait = 2, have_ks = 0;
    double h_ks = 0.0;
    memcpy(Z, tp->y0, sizeof(double) * n);
    rhs_r(pb, cell, tp->y0, f);
    for (int i = 0; i < n; ++i) Z[n + i] = tp->h0 * f[i];
    for (int r = 0; r < count && rc == 0; ++r) {
        const double *rec = tp->rec + (size_t)r * R;
        const double *P = rec + n, *c = rec + n + 36;
        const double gamma = rec[n + 42], il1 = rec[n + 43], h = rec[n + 46];
        const int q = (int)rec[n + 44], qo = (int)rec[n + 45];
        const int fails = (int)rec[n + 47] + (int)rec[n + 48];
        const int qin = r > 0 ? (int)tp->rec[(size_t)(r - 1) * R + n + 45] : 1;
        double *o = out + (size_t)r * 10;
        if ((int)rec[n + 48] >= 3) { qwait = 2; have_ks = 0; }
        else if (q < qin) qwait = q + 1;
        set_weights(n, Z, rtol, atol, w);                 /* from y_{n-1} */
        for (int a = 0; a < 6; ++a)
            for (int i = 0; i < n; ++i) {
                double sacc = 0.0;
                for (int b = 0; b < 6; ++b) sacc += P[a * 6 + b] * Z[b * n + i];
                Zp[a * n + i] = sacc;
            }
        predict(q, n, Zp);
        double xi[QMAX + 2], l[QMAX + 2], hist[QMAX + 1] = {0};
        for (int k = 0; k < QMAX && k < r; ++k) hist[k] = tp->rec[(size_t)(r - 1 - k) * R + n + 46];
        bdf_xi(q + 1, h, hist, xi);
        orc_bdf_l(q, xi, l);
        const double Cq = error_constant(l[1], xi[q]);
        for (int i = 0; i < n; ++i) d[i] = rec[i] - Zp[i];     /* Delta of the recorded state */
        o[0] = Cq * wrms(n, d, w);
        memcpy(ystar, Zp, sizeof(double) * n);
        if (exact_corrector(pb, cell, Zp, gamma, il1, ystar)) { rc = -2; break; }
        for (int i = 0; i < n; ++i) tmp2[i] = rec[i] - ystar[i];
        o[1] = Cq * wrms(n, tmp2, w);
        for (int i = 0; i < n; ++i) tmp2[i] = ystar[i] - Zp[i];
        o[6] = Cq * wrms(n, tmp2, w);
        o[7] = eta_from(o[6], q, 6.0);
        o[9] = fails;
        /* the corrected array (for the order q-1 estimate), then the choice */
        for (int j = 0; j <= q; ++j)
            for (int i = 0; i < n; ++i) zc[j * n + i] = Zp[j * n + i] + l[j] * d[i];
        if (r == count - 1) {
            o[2] = o[3] = o[4] = o[5] = NAN;
            o[8] = 0.0;
        } else {
            qwait--;
            const double etamax = fails ? 1.0 : (r == 0 ? 1e4 : 10.0);
            int newq;
            o[2] = choose_step(n, q, qmax, qwait, zc, d, w, xi, l, o[0], have_ks, ksave, h, h_ks, etamax,
                               tmp2, &newq);
            o[3] = newq;
            o[8] = qwait == 0;
            const double *nx = tp->rec + (size_t)(r + 1) * R;
            const int nfail = (int)nx[n + 47] + (int)nx[n + 48];
            o[4] = (nfail == 0 && r + 1 < count - 1) ? nx[n + 46] / h : NAN;
            o[5] = qo == q + 1 ? (double)(q + 1) : (nfail == 0 ? nx[n + 44] : NAN);
            /* the counter as the integrator leaves it (the recorded choice) */
            if (qo == q + 1 || qwait == 0) { qwait = qo + 1; have_ks = 0; }
            if (qwait == 1 && q < qmax) {
                const double kfac = l[1] * l[q] / (1.0 + l[1] * xi[q]);
                for (int i = 0; i < n; ++i) ksave[i] = kfac * d[i];
                h_ks = h; have_ks = 1;
            }
        }
        /* Z_n = Z_pred + c (y_n - z0_pred), columns above q_out zero */
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i < n; ++i)
                Z[j * n + i] = (j <= qo) ? ((j <= q ? Zp[j * n + i] : 0.0) + c[j] * d[i]) : 0.0;
    }
    free(Z); free(Zp); free(w); free(d); free(ystar); free(tmp2); free(ksave); free(f); free(zc);
    return rc;
}

/* Squared-error loss sum_k (Y_k - target_k)^2 at the replayed final state,
 * per cell in parallel: integrate with a tape, replay, adjoint.  yrep
 * [C, n], grad [C, M, 2]; returns the number of cells that failed. */
EXPORT int orc_adjoint_sqerr(const orc_problem *pb, long ncells, const double *y0,
                             const double *target, double t0, double tout,
                             const orc_options *op, int cap, double *yrep, double *grad,
                             int nthreads)
{
    int nbad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad)
    for (long c = 0; c < ncells; ++c) {
        const int n = pb->n, K = pb->K;
        orc_tape *tp = orc_tape_new(n, cap);
        double *y = malloc(sizeof(double) * n), *dL = malloc(sizeof(double) * n);
        memcpy(y, y0 + (size_t)c * n, sizeof(double) * n);
        int bad = bdf_cell(pb, c, y, t0, tout, op, NULL, NULL, tp) != 0 || tp->overflow;
        if (!bad) bad = orc_replay_tape(pb, c, tp, yrep + (size_t)c * n) != 0;
        if (!bad) {
            for (int i = 0; i < n; ++i)
                dL[i] = i < K ? 2.0 * (yrep[(size_t)c * n + i] - target[(size_t)c * K + i]) : 0.0;
            bad = orc_adjoint_tape(pb, c, tp, dL, grad + (size_t)c * 2 * pb->M) != 0;
        }
        nbad += bad;
        free(y); free(dL);
        orc_tape_free(tp);
    }
    return nbad;
}
