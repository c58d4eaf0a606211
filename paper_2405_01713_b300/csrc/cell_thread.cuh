// Thread-per-cell backend for very small systems (N <= 3): Robertson
// kinetics and the one-unknown heating-cooling cells.  All vectors, the
// Newton matrix and its pivots live in registers (every loop is unrolled at
// compile time; runtime indices select through predicates).
#pragma once
#include "sunb_common.cuh"
#include "erk_control.cuh"

namespace sunb {

// Robertson kinetics: y1' = -k1 y1 + k3 y2 y3, y2' = k1 y1 - k3 y2 y3 - k2 y2^2,
// y3' = k2 y2^2; parameters (k1, k2, k3) per cell.
struct RobertsonProblem {
    static constexpr int N = 3;
    double k1, k2, k3;
    __device__ void load(const double *params, int64_t cell)
    {
        k1 = params[3 * cell + 0];
        k2 = params[3 * cell + 1];
        k3 = params[3 * cell + 2];
    }
    __device__ __forceinline__ void rhs(const double *y, double *f) const
    {
        const double r1 = k1 * y[0], r2 = k2 * y[1] * y[1], r3 = k3 * y[1] * y[2];
        f[0] = -r1 + r3;
        f[1] = r1 - r3 - r2;
        f[2] = r2;
    }
    __device__ __forceinline__ void jac(const double *y, double (*J)[3]) const
    {
        J[0][0] = -k1;  J[0][1] = k3 * y[2];                     J[0][2] = k3 * y[1];
        J[1][0] = k1;   J[1][1] = -k3 * y[2] - 2.0 * k2 * y[1];  J[1][2] = -k3 * y[1];
        J[2][0] = 0.0;  J[2][1] = 2.0 * k2 * y[1];               J[2][2] = 0.0;
    }
    static constexpr bool kFusedJac = false;   // J costs extra work: only at set-ups
    // small batches spread about two cells per warp: evaluating the
    // order-q factor for every cell would add latency (+10 % measured)
    static constexpr bool kSharedEtaQ = false;
    // all Newton iterations of an attempt in one superstep (a cap of two
    // cost the spread batches 2 %)
    static constexpr int kNewtonPerSuperstep = MAXCOR;
    // cells of a one-wave launch all begin together: the start stays inline
    static constexpr bool kFoldedStart = false;
    // a failed attempt subtracts the prediction back out (a saved copy of
    // three-component columns would cost 36 registers)
    static constexpr bool kSavedPrediction = false;
};

// Cooling table in shared memory: knots lnT[i], values lnLam[i] and the
// per-segment log-log slopes.
struct CoolingSmem {
    int n;
    double gamma_heat;
    const double *lnT, *lnLam, *slope;
    const double *exptab;      // 2^(j/64), for fexp
    const float *lnTf;         // lnT rounded to float, for the knot search
};

// Heating-cooling of one gas cell (the Nyx split equation of Sec. 3.2,
// Eq. nyxODE): T = max(e, 1 K), de/dt = F + rho (Gamma (T/1e4)^-0.7 - Lambda(T)),
// Lambda piecewise power law through the knots (end slopes extended).
struct CosmologyProblem {
    static constexpr int N = 1;
    double rho, F;
    const CoolingSmem *tab;
    __device__ void load(const double *params, int64_t cell)
    {
        rho = params[2 * cell + 0];
        F = params[2 * cell + 1];
    }
    __device__ __forceinline__ void eval(double e, double &f, double &dfde) const
    {
        const bool floor = e < 1.0;
        const double T = floor ? 1.0 : e;
        const double lnT = flog(T);
        const double *x = tab->lnT;
        const int n = tab->n;
        // segment lo = the last knot i <= n - 2 with x[i] <= lnT (0 below
        // the first knot): a binary search on the float copy of the knots
        // (the FP32 pipe), then exact FP64 comparisons that move lo across
        // any knot the rounding to float put on the wrong side of lnT
        const float *xf = tab->lnTf;
        const float lf = (float)lnT;
        int lo;
        if (lf <= xf[0]) lo = 0;
        else if (lf >= xf[n - 1]) lo = n - 2;
        else {
            lo = 0;
            int hi = n - 1;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (xf[mid] <= lf) lo = mid; else hi = mid;
            }
        }
        while (lo > 0 && !(x[lo] <= lnT)) --lo;
        while (lo < n - 2 && x[lo + 1] <= lnT) ++lo;
        const double sl = tab->slope[lo];
        // Every rounding is spelled out (fma, or __dmul_rn, which is never
        // merged into a multiply-add): where a sum of products leaves the
        // compiler a choice of which product to fuse, or a product feeds two
        // sums, the choice may differ between the kernels that integrate
        // cosmology cells, and a cell's result would depend on which kernel
        // took it.
        const double lam = fexp(fma(sl, lnT - x[lo], tab->lnLam[lo]), tab->exptab);
        const double heat = __dmul_rn(tab->gamma_heat, fexp(-0.7 * (lnT - LN1E4), tab->exptab));
        f = fma(rho, heat - lam, F);
        dfde = floor ? 0.0 : rho * fma(-0.7, heat, -(sl * lam)) * rcp(T);
    }
    __device__ __forceinline__ void rhs(const double *y, double *f) const
    {
        double d;
        eval(y[0], f[0], d);
    }
    __device__ __forceinline__ void jac(const double *y, double (*J)[1]) const
    {
        double f;
        eval(y[0], f, J[0][0]);
    }
    // f and df/de come from one evaluation
    static constexpr bool kFusedJac = true;
    // full warps of cells: one shared evaluation of the order-q factor (-5 %)
    static constexpr bool kSharedEtaQ = true;
    // at most two Newton iterations per superstep: a warp no longer waits
    // for its slowest cell's third iteration, which runs in the next
    // superstep beside the other cells' first ones (-2.4 %; one per
    // superstep was 23 % slower: the control phases diverge)
    static constexpr int kNewtonPerSuperstep = 2;
    // a cell's start shares its warp's f evaluations (CellRun::begin_folded):
    // queue-fed warps begin cells at different supersteps
    static constexpr bool kFoldedStart = true;
    // a failed attempt restores the Nordsieck array saved before the
    // prediction (six doubles) instead of subtracting it back out: exact,
    // and no FP64 work on a path that some cell of a warp nearly always takes
    static constexpr bool kSavedPrediction = true;
    __device__ __forceinline__ void rhs_jac(const double *y, double *f, double (*J)[1]) const
    {
        eval(y[0], f[0], J[0][0]);
    }
};

// The step history of a thread-per-cell cell (REC = true, a separate
// kernel): states and control decisions in the tape layout of the lane-group
// backend (tape_header / tape_record doubles), without column maps (NaN).
template <bool REC> struct ThreadTape {
    __device__ __forceinline__ void rec_init(const double *, int, double) {}
    __device__ __forceinline__ void rec_accept(const double *, int, int, int, const double *, double, double,
                                               double, double, int, int) {}
};
template <> struct ThreadTape<true> {
    double *tape = nullptr;
    int tape_cap = 0, rec_count = 0;
    __device__ void rec_init(const double *y0, int N, double h0)
    {
        tape[0] = 0.0;
        tape[1] = h0;
        tape[2] = 0.0;
        for (int i = 0; i < N; ++i) tape[8 + i] = y0[i];   // y0 after the 8 header values
        rec_count = 0;
    }
    __device__ void rec_accept(const double *y, int N, int q, int qo, const double *l, double inv_xi, double gamma,
                               double il1, double h, int ncf, int nef)
    {
        if (rec_count >= tape_cap) {
            tape[2] = 1.0;
            return;
        }
        double *r = tape + tape_header(N) + (size_t)rec_count * tape_record(N);
        for (int i = 0; i < N; ++i) r[i] = y[i];
        for (int i = 0; i < 36; ++i) r[N + i] = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            double c = (j <= q) ? l[j] : 0.0;
            if (qo == q + 1 && j >= 1 && j <= q + 1) c += l[j - 1] * inv_xi;
            r[N + 36 + j] = c;
        }
        r[N + 42] = gamma;
        r[N + 43] = il1;
        r[N + 44] = (double)q;
        r[N + 45] = (double)qo;
        r[N + 46] = h;
        r[N + 47] = (double)ncf;
        r[N + 48] = (double)nef;
        tape[0] = (double)(++rec_count);
    }
};

template <class Prob, bool REC = false>
struct ThreadCell : ThreadTape<REC> {
    static constexpr int N = Prob::N;
    // Newton iterations per superstep (the problem's choice): most or all
    // of an attempt's, so that the control logic (cheap f, costly control)
    // stays aligned across the warp
    static constexpr int kNewtonPerSuperstep = Prob::kNewtonPerSuperstep;
    static constexpr bool kOutlineRare = false;
    // the order-q step factor evaluated once before the error test's branch
    // (see CellRun::post) where the problem's batches fill whole warps
    static constexpr bool kSharedEtaQ = Prob::kSharedEtaQ;
    static constexpr bool kFoldedStart = Prob::kFoldedStart;
    // linear solves with the LU factors (no Krylov variant)
    static constexpr bool kKrylov = false;
    Prob prob;
    double v[NVEC][N];
    double zs[Prob::kSavedPrediction ? QMAX + 1 : 1][N];   // the array before predict()
    double M[N][N];
    double atol[N];
    double *yg;   // this cell's state in global memory

    __device__ __forceinline__ void rec_init(double h0) { ThreadTape<REC>::rec_init(v[V_Z0], N, h0); }
    __device__ __forceinline__ void rec_accept(int q, int qo, const double *l, double inv_xi, double gamma,
                                               double il1, double h, int ncf, int nef)
    {
        ThreadTape<REC>::rec_accept(v[V_Z0], N, q, qo, l, inv_xi, gamma, il1, h, ncf, nef);
    }

    __device__ __forceinline__ void load_y(int s)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[s][i] = yg[i];
    }
    __device__ __forceinline__ void store_y(int s)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) yg[i] = v[s][i];
    }
    __device__ __forceinline__ void rhs(int a, int b) { prob.rhs(v[a], v[b]); }
    __device__ __forceinline__ void rhs_start(int a, int b) { prob.rhs(v[a], v[b]); }
    __device__ __forceinline__ bool all_finite(int a) const
    {
        bool ok = true;
#pragma unroll
        for (int i = 0; i < N; ++i) ok = ok && (fabs(v[a][i]) <= 1.7e308);
        return ok;
    }
    __device__ __forceinline__ void set_weights(int a, double rtol)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[V_W][i] = rcp(fma(rtol, fabs(v[a][i]), atol[i]));
    }
    // squared WRMS norm of slot a; a may be a runtime Nordsieck column
    __device__ __forceinline__ double wrms2(int a) const
    {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NVEC; ++j) {
            if (j == a) {
#pragma unroll
                for (int i = 0; i < N; ++i) { const double t = v[j][i] * v[V_W][i]; s += t * t; }
            }
        }
        return s * (1.0 / N);
    }
    // squared WRMS norm of the corrected column q, z_q + lq Delta, before
    // the correction is applied (q a runtime order, selected by predicate)
    __device__ __forceinline__ double wrms2_corrected(int q, double lq) const
    {
        double s = 0.0;
#pragma unroll
        for (int j = 1; j <= QMAX; ++j) {
            if (j == q) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const double t = fma(lq, v[V_ACOR][i], v[j][i]) * v[V_W][i];
                    s += t * t;
                }
            }
        }
        return s * (1.0 / N);
    }
    // (a x + b y with the product a x fused, in every kernel alike: the sum
    // of two products leaves the compiler a choice otherwise)
    __device__ __forceinline__ double wrms2_lin(double a, int va, double b, int vb) const
    {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double t = fma(a, v[va][i], b * v[vb][i]) * v[V_W][i];
            s += t * t;
        }
        return s * (1.0 / N);
    }
    __device__ __forceinline__ void axpby(int o, double a, int va, double b, int vb)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[o][i] = fma(b, v[vb][i], a * v[va][i]);   // b y fused
    }
    __device__ __forceinline__ void copy(int o, int va)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[o][i] = v[va][i];
    }
    __device__ __forceinline__ void scale(int o, double a, int va)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[o][i] = a * v[va][i];
    }
    __device__ __forceinline__ void predict(int q)
    {
        if constexpr (Prob::kSavedPrediction) {
#pragma unroll
            for (int j = 0; j <= QMAX; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) zs[j][i] = v[j][i];
        }
#pragma unroll
        for (int k = 0; k < QMAX; ++k)
#pragma unroll
            for (int j = QMAX; j >= 1; --j)
                if (k < q && j > k && j <= q)
#pragma unroll
                    for (int i = 0; i < N; ++i) v[j - 1][i] += v[j][i];
    }
    __device__ __forceinline__ void unpredict(int q)
    {
        if constexpr (Prob::kSavedPrediction) {
#pragma unroll
            for (int j = 0; j <= QMAX; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] = zs[j][i];
        } else {
#pragma unroll
            for (int k = QMAX - 1; k >= 0; --k)
#pragma unroll
                for (int j = 1; j <= QMAX; ++j)
                    if (k < q && j > k && j <= q)
#pragma unroll
                        for (int i = 0; i < N; ++i) v[j - 1][i] -= v[j][i];
        }
    }
    __device__ __forceinline__ void rescale(int q, double eta)
    {
        double f = 1.0;
#pragma unroll
        for (int j = 1; j <= QMAX; ++j) {
            f *= eta;
            if (j <= q)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] *= f;
        }
    }
    __device__ __forceinline__ void correct(int q, const double *l)
    {
#pragma unroll
        for (int j = 0; j <= QMAX; ++j)
            if (j <= q)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] = fma(l[j], v[V_ACOR][i], v[j][i]);
    }
    __device__ __forceinline__ void order_increase(int q, const double *l, double inv_xi)
    {
#pragma unroll
        for (int j = 1; j <= QMAX; ++j) {
            if (j == q + 1)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] = 0.0;
            if (j <= q + 1) {
                const double c = l[j - 1] * inv_xi;
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] += c * v[V_ACOR][i];
            }
        }
    }
    __device__ __forceinline__ void order_decrease(int q, const double *e)
    {
        double zq[N];
#pragma unroll
        for (int i = 0; i < N; ++i) zq[i] = 0.0;
#pragma unroll
        for (int j = 2; j <= QMAX; ++j)
            if (j == q)
#pragma unroll
                for (int i = 0; i < N; ++i) zq[i] = v[j][i];
#pragma unroll
        for (int j = 1; j < QMAX; ++j)
            if (j < q)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] -= e[j - 1] * zq[i];
#pragma unroll
        for (int j = 2; j <= QMAX; ++j)
            if (j == q)
#pragma unroll
                for (int i = 0; i < N; ++i) v[j][i] = 0.0;
    }
    __device__ __forceinline__ void restart(double h)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[1][i] = h * v[V_F][i];
#pragma unroll
        for (int j = 2; j <= QMAX; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) v[j][i] = 0.0;
    }
    __device__ __forceinline__ void newton_init()
    {
#pragma unroll
        for (int i = 0; i < N; ++i) { v[V_ACOR][i] = 0.0; v[V_Y][i] = v[V_Z0][i]; }
    }
    __device__ __forceinline__ void newton_residual(double h, double il1)
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
            v[V_DEL][i] = fma(fma(h, v[V_F][i], -v[V_Z1][i]), il1, -v[V_ACOR][i]);
    }
    __device__ __forceinline__ double newton_update(double c)
    {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double d = __dmul_rn(v[V_DEL][i], c);   // feeds two sums: never fused
            v[V_ACOR][i] += d;
            v[V_Y][i] = v[V_Z0][i] + v[V_ACOR][i];
            const double t = d * v[V_W][i];
            s += t * t;
        }
        return s * (1.0 / N);
    }
    // ---------------- explicit Runge-Kutta (ErkRun) ----------------
    // stage derivatives k_0..k_4 in slots 1..5; the stage index j is a
    // runtime value, so slots are selected through predicates
    __device__ __forceinline__ void erk_stage(int j, double h)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (m < j) s += ERK_A[j][m] * v[1 + m][i];
            v[V_Y][i] = v[V_Z0][i] + h * s;
        }
    }
    __device__ __forceinline__ void erk_rhs(int j)
    {
        double f[N];
        prob.rhs(v[V_Y], f);
#pragma unroll
        for (int m = 0; m < 5; ++m)
            if (m == j)
#pragma unroll
                for (int i = 0; i < N; ++i) v[1 + m][i] = f[i];
    }
    __device__ __forceinline__ double erk_error2(double h) const
    {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double e = 0.0;
#pragma unroll
            for (int m = 0; m < 5; ++m) e += (ERK_B[m] - ERK_BH[m]) * v[1 + m][i];
            const double t = (h * e) * v[V_W][i];
            s += t * t;
        }
        return s * (1.0 / N);
    }
    __device__ __forceinline__ void erk_accept(double h)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double sb = 0.0;
#pragma unroll
            for (int m = 0; m < 5; ++m) sb += ERK_B[m] * v[1 + m][i];
            v[V_Z0][i] += h * sb;
        }
    }

    __device__ __forceinline__ bool acquire_setup() { return true; }
    __device__ __forceinline__ int f_per_setup() const { return 0; }
    // the f evaluation of a Newton iteration, f(y) into V_F; with setup also
    // the Newton matrix at y, factored (0: singular)
    __device__ __forceinline__ int newton_f(bool setup, double gamma)
    {
        // where J comes with f (Prob::kFusedJac), one evaluation serves both,
        // so that cells of a warp that set up and cells that do not share it
        double J[N][N];
        if constexpr (Prob::kFusedJac) {
            prob.rhs_jac(v[V_Y], v[V_F], J);
            if (!setup) return 1;
        } else {
            prob.rhs(v[V_Y], v[V_F]);
            if (!setup) return 1;
            prob.jac(v[V_Y], J);
        }
        return factor_from(J, gamma);
    }
    // M = I - gamma J, in-register LU with row partial pivoting (first index
    // of largest magnitude).  Pivots are kept as an explicit permutation
    // applied in solve().
    int perm[N];
    __device__ __forceinline__ int factor_from(const double (*J)[N], double gamma)
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) M[i][j] = (i == j ? 1.0 : 0.0) - gamma * J[i][j];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < N; ++i) perm[i] = i;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            int p = k;
            double amax = fabs(M[k][k]);
#pragma unroll
            for (int i = k + 1; i < N; ++i)
                if (fabs(M[i][k]) > amax) { amax = fabs(M[i][k]); p = i; }
            ok = ok && (amax > 0.0) && (amax <= 1.7e308);
#pragma unroll
            for (int i = k + 1; i < N; ++i) {
                if (i == p) {
#pragma unroll
                    for (int j = 0; j < N; ++j) { const double t = M[k][j]; M[k][j] = M[i][j]; M[i][j] = t; }
                    const int tp = perm[k]; perm[k] = perm[i]; perm[i] = tp;
                }
            }
            const double ip = rcp(M[k][k]);
#pragma unroll
            for (int i = k + 1; i < N; ++i) {
                const double lik = M[i][k] * ip;
                M[i][k] = lik;
#pragma unroll
                for (int j = k + 1; j < N; ++j) M[i][j] -= lik * M[k][j];
            }
            M[k][k] = ip;     // keep the reciprocal pivot for the back solve
        }
        return ok ? 1 : 0;
    }
    __device__ __forceinline__ void solve(int b)
    {
        double x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) if (perm[i] == j) t = v[b][j];
            x[i] = t;
        }
#pragma unroll
        for (int i = 1; i < N; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j) x[i] -= M[i][j] * x[j];
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
#pragma unroll
            for (int j = i + 1; j < N; ++j) x[i] -= M[i][j] * x[j];
            x[i] *= M[i][i];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) v[b][i] = x[i];
    }
};

}  // namespace sunb
