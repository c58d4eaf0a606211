/* Right-hand sides of the oracle, written once and included twice by
 * oracle.c: with REAL = double (integration) and with REAL = double complex
 * (complex-step Jacobians, which differentiate these very functions).
 *
 * Test infrastructure only: nothing in the CUDA path includes this file.
 *
 * Before inclusion the includer defines
 *   REAL       the scalar type,
 *   FN(name)   the function-name decoration for this scalar type,
 *   RE(x)      the real part of x,
 *   EXPF/LOGF  exp and log for REAL.
 */

/* Robertson kinetics (the classic stiff test of chemical kinetics):
 *   y1' = -k1 y1 + k3 y2 y3,  y2' = k1 y1 - k3 y2 y3 - k2 y2^2,  y3' = k2 y2^2
 * with k = (k1, k2, k3) per cell. */
static void FN(rhs_robertson)(const double *k, const REAL *y, REAL *f)
{
    REAL r1 = k[0] * y[0];
    REAL r2 = k[1] * y[1] * y[1];
    REAL r3 = k[2] * y[1] * y[2];
    f[0] = -r1 + r3;
    f[1] = r1 - r3 - r2;
    f[2] = r2;
}

/* Constant-pressure adiabatic reactor: the chemical source term R of the
 * Pele split system dU/dt = F + R (Sec. 3.1, Eq. chemODE), written for the
 * state U = (Y_1..Y_K, T) at fixed pressure P:
 *   rho      = P Wbar / (Ru T),  1/Wbar = sum_k Y_k / W_k
 *   C_k      = rho Y_k / W_k                               (mol/cm^3)
 *   kf_j     = A_j T^b_j exp(-Ea_j / (Rc T))
 *   Kc_j     = exp(-dG_j/RT) (P_atm/(Ru T))^(dnu_j)
 *   q_j      = kf_j prod_reactants C - (kf_j/Kc_j) prod_products C
 *   wdot_k   = sum_j (nu''_kj - nu'_kj) q_j
 *   dY_k/dt  = wdot_k W_k / rho
 *   dT/dt    = -sum_k H_k wdot_k / (rho cp),  H_k = Ru T (h/RT)_k,
 *              cp = Ru sum_k Y_k (cp/R)_k / W_k
 * with single-range NASA-7 polynomials for cp/R, h/RT and s/R.  With
 * only >= 0, wdot keeps reaction `only` alone (f is linear in the rates of
 * progress, so this is d f / d ln A_only). */
static void FN(rhs_mechanism)(const orc_problem *pb, const double *prm,
                              const REAL *y, REAL *f, int only)
{
    const int K = pb->K, M = pb->M;
    const double P = prm[0];
    REAL T = y[K];
    REAL lnT = LOGF(T);
    REAL sumYW = 0.0;
    for (int k = 0; k < K; ++k) sumYW += y[k] / pb->W[k];
    REAL rho = P / (ORC_RU * T * sumYW);

    REAL C[K], hRT[K], gRT[K], cpR[K], wdot[K];
    REAL T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    for (int k = 0; k < K; ++k) {
        const double *a = pb->nasa + 7 * k;
        C[k] = rho * y[k] / pb->W[k];
        cpR[k] = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
        hRT[k] = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0
               + a[4] * T4 / 5.0 + a[5] / T;
        REAL sR = a[0] * lnT + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0
                + a[4] * T4 / 4.0 + a[6];
        gRT[k] = hRT[k] - sR;
        wdot[k] = 0.0;
    }
    REAL patm_RT = ORC_PATM / (ORC_RU * T);
    for (int j = 0; j < M; ++j) {
        if (only >= 0 && j != only) continue;   /* one reaction's share of wdot */
        const int *r = pb->react + 3 * j, *p = pb->prod + 3 * j;
        REAL kf = EXPF(pb->lnA[j] + pb->beta[j] * lnT - pb->Ea[j] / (ORC_RC * T));
        REAL dG = 0.0;
        int dnu = 0;
        REAL fwd = kf, rev = 1.0;
        for (int s = 0; s < 3; ++s) {
            if (r[s] >= 0) { dG -= gRT[r[s]]; dnu -= 1; fwd *= C[r[s]]; }
            if (p[s] >= 0) { dG += gRT[p[s]]; dnu += 1; rev *= C[p[s]]; }
        }
        REAL Kc = EXPF(-dG);
        for (int i = 0; i < dnu; ++i) Kc *= patm_RT;
        for (int i = 0; i < -dnu; ++i) Kc /= patm_RT;
        REAL q = fwd - (kf / Kc) * rev;
        for (int s = 0; s < 3; ++s) {
            if (r[s] >= 0) wdot[r[s]] -= q;
            if (p[s] >= 0) wdot[p[s]] += q;
        }
    }
    REAL cp = 0.0, hw = 0.0;
    for (int k = 0; k < K; ++k) {
        f[k] = wdot[k] * pb->W[k] / rho;
        cp += y[k] * cpR[k] / pb->W[k];
        hw += hRT[k] * wdot[k];
    }
    cp *= ORC_RU;
    f[K] = -(ORC_RU * T * hw) / (rho * cp);
}

/* Heating-cooling of one gas cell, the Nyx split equation de/dt = F + R
 * (Sec. 3.2, Eq. nyxODE), with T = e and
 *   R = rho (Gamma (T/1e4)^-0.7 - Lambda(T)),
 * Lambda a piecewise power law through the tabulated knots (linear in
 * log-log, extended past either end with the end segment's slope).  The
 * temperature is floored at 1 K inside R, so that Newton iterates that dip
 * below zero stay finite.  prm = (rho, F). */
static void FN(rhs_cosmology)(const orc_problem *pb, const double *prm,
                              const REAL *y, REAL *f)
{
    REAL T = y[0];
    if (RE(T) < 1.0) T = 1.0;
    REAL lnT = LOGF(T);
    const double *x = pb->lnT, *v = pb->lnLam;
    int n = pb->nknots;
    /* segment i with x[i] <= lnT < x[i+1], clamped to the end segments */
    int lo = 0, hi = n - 1;
    double lt = RE(lnT);
    if (lt <= x[0]) { lo = 0; }
    else if (lt >= x[n - 1]) { lo = n - 2; }
    else {
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (x[mid] <= lt) lo = mid; else hi = mid;
        }
    }
    double slope = (v[lo + 1] - v[lo]) / (x[lo + 1] - x[lo]);
    REAL lam = EXPF(v[lo] + slope * (lnT - x[lo]));
    REAL heat = pb->gamma_heat * EXPF(-0.7 * (lnT - ORC_LN1E4));
    f[0] = prm[1] + prm[0] * (heat - lam);
}

/* Linear constant-coefficient system y' = A y, A per cell (row-major). */
static void FN(rhs_linear)(const orc_problem *pb, const double *A,
                           const REAL *y, REAL *f)
{
    int n = pb->n;
    for (int i = 0; i < n; ++i) {
        REAL s = 0.0;
        for (int j = 0; j < n; ++j) s += A[i * n + j] * y[j];
        f[i] = s;
    }
}

static void FN(rhs)(const orc_problem *pb, long cell, const REAL *y, REAL *f)
{
    const double *prm = pb->params + (size_t)cell * pb->nparams;
    switch (pb->kind) {
    case ORC_ROBERTSON: FN(rhs_robertson)(prm, y, f); break;
    case ORC_MECHANISM: FN(rhs_mechanism)(pb, prm, y, f, -1); break;
    case ORC_COSMOLOGY: FN(rhs_cosmology)(pb, prm, y, f); break;
    case ORC_LINEAR:    FN(rhs_linear)(pb, prm, y, f); break;
    }
}
