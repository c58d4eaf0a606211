// Group-of-lanes-per-cell backend for reaction mechanisms (N = K + 1 up to
// 64 unknowns): L lanes (8, 16 or 32) serve one cell, several cells share a
// warp when L < 32.  The Nordsieck history, the Newton vectors, the Newton
// matrix and the right-hand-side scratch of each cell live in shared memory
// ("CY" order, Sec. 4.1.2: all components of a cell contiguous, so the
// per-cell Jacobian is a dense block); the mechanism tables are staged once
// per CTA.  Group reductions are butterfly shuffles within the L lanes, so
// every result is deterministic.
//
// Right-hand side: the chemical source term R of Eq. chemODE (Sec. 3.1) for
// a constant-pressure adiabatic reactor, y = (Y_1..Y_K, T):
//   rho = P/(Ru T sum_k Y_k/W_k),  C_k = rho Y_k / W_k,
//   kf_j = exp(ln A_j + b_j ln T - (Ea_j/Rc)/T),
//   kr_j = kf_j / Kc_j,  Kc_j = exp(-dG_j/RT) (P_atm/(Ru T))^dnu_j,
//   q_j = kf_j prod_reac C - kr_j prod_prod C,  wdot_k = sum_j nu_kj q_j,
//   dY_k/dt = W_k wdot_k / rho,  dT/dt = -T sum_k (h/RT)_k wdot_k / (rho sum_k Y_k (cp/R)_k / W_k).
// exp(-dG/RT) is formed as a product of per-species factors exp(+-g_k),
// g_k = (h/RT)_k - (s/R)_k, which needs K exponentials instead of M.
//
// Analytic Jacobian (Table 1, "Analytical"; the paper's Sec. 4.1.4 finds it
// faster than difference quotients).  With Jc = d wdot / d C at fixed T,
// u = Jc C, Wbar/rho = Ru T / P:
//   J_kl = (W_k/W_l) (Jc_kl + (Ru T/P)(wdot_k - u_k))
//   J_kT = (W_k/rho) (dwdot_k/dT|_C + (wdot_k - u_k)/T)
//   J_Tl = -(1/(W_l cpm)) (T (S_l - (Ru T/P) U) + f_T ((cp/R)_l - cpm Wbar))
//   J_TT = -(sum_k (cp/R)_k wdot_k + T sum_k (h/RT)_k (dwdot_k/dT|_C - u_k/T)) / (rho cpm)
//          - f_T (-1/T + sum_k Y_k (dcp/R/dT)_k / W_k / cpm)
// with S_l = sum_k (h/RT)_k Jc_kl, U = sum_k (h/RT)_k u_k, cpm = sum_k Y_k (cp/R)_k/W_k.
// The matrix is built pre-multiplied by gamma, so M = I - gamma J directly,
// in precision MT (double, or float for the mixed form).
#pragma once
#include "sunb_common.cuh"

namespace sunb {

// Byte offsets of the mechanism tables inside the staged blob.
struct MechTabOffsets {
    int K, M, N, nnz;
    int invW, W, cpc, hc, sc, dcp, rpar, atol, inc_nu;   // double arrays
    int ridx, inc_ptr, inc_j, inc_nuf, invWf;            // 32-bit arrays
    int exptab;                                          // the exp table (EXP_TABLE_SIZE doubles)
    int bytes;                                           // blob size (multiple of 16)
};

// Per-cell shared-memory layout (byte offsets from the cell's base; dq < 0:
// the Newton-matrix scratch lives outside the cell and is set by
// set_jac_scratch, pm < 0: no adjoint map).
struct CellLayout {
    int NP;            // padded vector length
    int vec, mat, perm, xs, sp, rq, dq, pm, bytes;   // xs: 2N MT (solve scratch, reciprocal pivots);
                                                     // pm: 36 + K + 1 doubles (adjoint map and scratch)
};

struct MechTab {
    int K, M, N;
    const double *invW, *W, *cpc, *hc, *sc, *dcp, *rpar, *atol, *inc_nu;
    const uint32_t *ridx;
    const int32_t *inc_ptr, *inc_j;
    const float *inc_nuf, *invWf;          // FP32 copies for the FP32 Newton matrix
    const double *exptab;                  // 2^(j/64), for fexp
    template <typename T> __device__ __forceinline__ const T *nu() const;
    template <typename T> __device__ __forceinline__ const T *iw() const;
};
template <> __device__ __forceinline__ const double *MechTab::nu<double>() const { return inc_nu; }
template <> __device__ __forceinline__ const float *MechTab::nu<float>() const { return inc_nuf; }
template <> __device__ __forceinline__ const double *MechTab::iw<double>() const { return invW; }
template <> __device__ __forceinline__ const float *MechTab::iw<float>() const { return invWf; }

__device__ __forceinline__ MechTab mech_tab_at(const unsigned char *base, const MechTabOffsets &o)
{
    MechTab t;
    t.K = o.K; t.M = o.M; t.N = o.N;
    t.invW = reinterpret_cast<const double *>(base + o.invW);
    t.W = reinterpret_cast<const double *>(base + o.W);
    t.cpc = reinterpret_cast<const double *>(base + o.cpc);
    t.hc = reinterpret_cast<const double *>(base + o.hc);
    t.sc = reinterpret_cast<const double *>(base + o.sc);
    t.dcp = reinterpret_cast<const double *>(base + o.dcp);
    t.rpar = reinterpret_cast<const double *>(base + o.rpar);
    t.atol = reinterpret_cast<const double *>(base + o.atol);
    t.inc_nu = reinterpret_cast<const double *>(base + o.inc_nu);
    t.ridx = reinterpret_cast<const uint32_t *>(base + o.ridx);
    t.inc_ptr = reinterpret_cast<const int32_t *>(base + o.inc_ptr);
    t.inc_j = reinterpret_cast<const int32_t *>(base + o.inc_j);
    t.inc_nuf = reinterpret_cast<const float *>(base + o.inc_nuf);
    t.invWf = reinterpret_cast<const float *>(base + o.invWf);
    t.exptab = reinterpret_cast<const double *>(base + o.exptab);
    return t;
}

template <int L>
struct Grp {
    int lane;
    unsigned mask;
    __device__ __forceinline__ double sum(double v) const
    {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
        return v;
    }
    __device__ __forceinline__ double max(double v) const
    {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
        return v;
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

template <typename MT> __device__ __forceinline__ MT mt_rcp(MT x);
template <> __device__ __forceinline__ double mt_rcp<double>(double x) { return __drcp_rn(x); }
template <> __device__ __forceinline__ float mt_rcp<float>(float x) { return __frcp_rn(x); }


// ---------------- dense LU with row partial pivoting (Sec. 4.1.4, 4.1.6) ----
// L lanes factor one N x N row-major matrix in place: unit-lower multipliers
// below the diagonal, U on and above it.  Pivot = first row of largest
// magnitude (ties to the lower index).  perm[i] is the original row of
// factored row i; piv (optional) receives the LAPACK-style exchange sequence;
// dinv[k] = 1/U_kk.  The rank-1 updates spread the (N-k-1)^2 entries over
// all L lanes.  Returns 1, or 0 if a pivot is zero or not finite.
template <int L, typename MT>
__device__ int lu_factor(const Grp<L> &g, MT *mat, int N, int32_t *perm, MT *dinv, int32_t *piv)
{
    int ok = 1;
    for (int i = g.lane; i < N; i += L) perm[i] = i;
    g.sync();
    for (int k = 0; k < N; ++k) {
        MT best = (MT)-1;
        int bi = N;
        for (int i = k + g.lane; i < N; i += L) {
            const MT a = fabs(mat[i * N + k]);
            if (a > best) { best = a; bi = i; }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            const MT ob = __shfl_xor_sync(g.mask, best, o);
            const int oi = __shfl_xor_sync(g.mask, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        ok = ok && (best > (MT)0) && (best <= (MT)3.0e38);
        const int p = (bi < N) ? bi : k;
        if (p != k) {
            for (int j = g.lane; j < N; j += L) {
                const MT t = mat[k * N + j];
                mat[k * N + j] = mat[p * N + j];
                mat[p * N + j] = t;
            }
        }
        if (g.lane == 0) {
            if (p != k) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
            if (piv) piv[k] = p;
        }
        g.sync();
        const MT ip = mt_rcp<MT>(mat[k * N + k]);
        for (int i = k + 1 + g.lane; i < N; i += L) mat[i * N + k] *= ip;
        if (g.lane == 0) dinv[k] = ip;
        g.sync();
        const int m = N - k - 1;
        if (m > 0) {
            const int total = m * m;
            const int di = L / m, dj = L % m;
            int ii = g.lane / m, jj = g.lane % m;
            for (int e = g.lane; e < total; e += L) {
                MT *r = mat + (k + 1 + ii) * N;
                r[k + 1 + jj] -= r[k] * mat[k * N + k + 1 + jj];
                ii += di; jj += dj;
                if (jj >= m) { jj -= m; ++ii; }
            }
        }
        g.sync();
    }
    return ok;
}

// Solve with the factors of lu_factor: b (length N, type BT) is overwritten
// by the solution; the arithmetic runs in MT with scratch xs.
template <int L, typename MT, typename BT>
__device__ void lu_solve(const Grp<L> &g, const MT *mat, int N, const int32_t *perm,
                         const MT *dinv, MT *xs, BT *b)
{
    for (int i = g.lane; i < N; i += L) xs[i] = (MT)b[perm[i]];
    g.sync();
    for (int k = 0; k < N - 1; ++k) {
        const MT xk = xs[k];
        for (int i = k + 1 + g.lane; i < N; i += L) xs[i] -= mat[i * N + k] * xk;
        g.sync();
    }
    for (int k = N - 1; k >= 0; --k) {
        const MT xk = xs[k] * dinv[k];
        for (int i = g.lane; i < k; i += L) xs[i] -= mat[i * N + k] * xk;
        g.sync();
        if (g.lane == 0) xs[k] = xk;
        g.sync();
    }
    for (int i = g.lane; i < N; i += L) b[i] = (BT)xs[i];
    g.sync();
}

// Solve M^T x = b with the factors of lu_factor (P M = L U, so
// M^T = U^T L^T P): U^T w = b, L^T v = w, x_perm[i] = v_i.  In place in b.
template <int L>
__device__ void lu_solve_t(const Grp<L> &g, const double *mat, int N, const int32_t *perm,
                           const double *dinv, double *xs, double *b)
{
    for (int i = g.lane; i < N; i += L) xs[i] = b[i];
    g.sync();
    for (int k = 0; k < N; ++k) {
        const double wk = xs[k] * dinv[k];
        for (int i = k + 1 + g.lane; i < N; i += L) xs[i] -= mat[k * N + i] * wk;
        g.sync();
        if (g.lane == 0) xs[k] = wk;
        g.sync();
    }
    for (int k = N - 1; k > 0; --k) {
        const double vk = xs[k];
        for (int i = g.lane; i < k; i += L) xs[i] -= mat[k * N + i] * vk;
        g.sync();
    }
    for (int i = g.lane; i < N; i += L) b[perm[i]] = xs[i];
    g.sync();
}


// Krylov scratch of one lane group (global memory, doubles): the basis
// [l+1][N], the Hessenberg matrix [l+1][l], the rotations cs and sn [l],
// the rotated right side [l+1], the solution coefficients [l], and the
// perturbed state and its f [N] each, for the Krylov dimension
// l = min(N, KRYLOV_MAXL) (no restarts).
constexpr int KRYLOV_MAXL = 64;
__host__ __device__ __forceinline__ int krylov_dim(int N) { return N < KRYLOV_MAXL ? N : KRYLOV_MAXL; }
__host__ __device__ __forceinline__ int krylov_doubles(int N)
{
    const int l = krylov_dim(N);
    return ((l + 1) * N + (l + 1) * l + 4 * l + 1 + 2 * N + 3) & ~3;
}

// the GMRES scratch pointer, a member of the Krylov variant only (an empty
// base of the direct one, which so keeps its layout)
template <bool KRY> struct KrylovScratch {};
template <> struct KrylovScratch<true> { double *kry = nullptr; };   // krylov_doubles(N) of this group

template <int L, typename MT, bool KRY = false>
struct GroupCell : KrylovScratch<KRY> {
    // one Newton iteration per superstep: a group that needs another
    // iteration takes it in the next superstep, at the same f call site as
    // the first iterations of the other groups of its warp
    static constexpr int kNewtonPerSuperstep = 1;
    // the starting step and the failure paths out of line (see CellRun)
    static constexpr bool kOutlineRare = true;
    // the order-q step factor only where a path needs it (see CellRun::post)
    static constexpr bool kSharedEtaQ = false;
    // cells begin through begin_body (out of line): a lane group's start
    // evaluations are group-wide calls of their own
    static constexpr bool kFoldedStart = false;
    // matrix-free GMRES linear solves in the scratch kry instead of LU
    // factors (a separate kernel, so the direct kernel carries none of it)
    static constexpr bool kKrylov = KRY;
    Grp<L> g;
    MechTab tb;
    int N, K, M, NP;
    double invN, P, invP;
    double *vec;          // [NVEC][NP]
    MT *mat;              // [N][N], row-major
    int32_t *perm;        // [N] row permutation of the factorisation
    MT *xs;               // [N] solve scratch
    MT *dinv;             // [N] reciprocal pivots
    double *C, *D, *egi, *hRT, *cpR;                    // species scratch ([K+1] for the first four);
                                                        // D_k = exp(g_k) C_k, egi_k = exp(-g_k)
    double *wdot, *u, *wT;                              // [K] each, Newton-matrix builds only
    double *q;                                          // [M]
    MT *dq;                                             // [6M] gamma dq_j/dC at each position
    double *dqdT, *uq;                                  // [M] gamma dq_j/dT, gamma sum_m C_m dq_j/dC_m
    double *yg;
    int *jac_lock = nullptr;   // non-null: dq/dqdT/uq shared with the other groups of the warp
    bool jac_dq = false;       // Newton matrix from difference quotients instead of the analytic J
    // discrete-adjoint recording (null tape: no recording)
    double *tape = nullptr;
    int tape_cap = 0, rec_count = 0;
    double *Pm;          // [36] column map accumulated since the last accepted step
    double *wmu;         // [K+1] adjoint scratch (W_k mu_k, zero sentinel)
    double last_rho, last_cpm, last_T;

    __device__ __forceinline__ double *V(int s) const { return vec + s * NP; }

    __device__ void bind(unsigned char *base, const CellLayout &lay)
    {
        NP = lay.NP;
        vec = reinterpret_cast<double *>(base + lay.vec);
        mat = reinterpret_cast<MT *>(base + lay.mat);
        perm = reinterpret_cast<int32_t *>(base + lay.perm);
        xs = reinterpret_cast<MT *>(base + lay.xs);
        dinv = xs + N;
        double *sp = reinterpret_cast<double *>(base + lay.sp);
        C = sp; D = C + (K + 1); egi = D + (K + 1); hRT = egi + (K + 1);
        cpR = hRT + (K + 1);
        q = reinterpret_cast<double *>(base + lay.rq);
        if (lay.dq >= 0) set_jac_scratch(base + lay.dq, nullptr);
        if (lay.pm >= 0) {
            Pm = reinterpret_cast<double *>(base + lay.pm);
            wmu = Pm + 36;
        } else {
            Pm = wmu = nullptr;
        }
        if (g.lane == 0) {
            C[K] = 1.0; D[K] = 1.0; egi[K] = 1.0; hRT[K] = 0.0;
            if (wmu) wmu[K] = 0.0;
        }
        g.sync();
    }

    // Newton-matrix scratch: dq [6M] in MT, then dqdT and uq [M] and wdot,
    // u, wT [K] in FP64 (jac_scratch_bytes).  With a lock, the groups of a
    // warp share one
    // scratch: a group takes it before a set-up (acquire_setup) and gives
    // it back once its matrix is assembled, within one superstep, so no
    // group ever waits for it.
    __device__ void set_jac_scratch(unsigned char *p, int *lock)
    {
        dq = reinterpret_cast<MT *>(p);
        dqdT = reinterpret_cast<double *>(p + ((6 * M * (int)sizeof(MT) + 15) & ~15));
        uq = dqdT + M;
        wdot = uq + M;
        u = wdot + K;
        wT = u + K;
        jac_lock = lock;
    }
    __device__ __forceinline__ bool acquire_setup()
    {
        if (!jac_lock) return true;
        int got = 0;
        if (g.lane == 0) got = (atomicCAS(jac_lock, 0, 1) == 0);
        return __shfl_sync(g.mask, got, 0, L) != 0;
    }
    __device__ __forceinline__ void release_setup()
    {
        if (!jac_lock) return;
        g.sync();
        if (g.lane == 0) {
            __threadfence_block();
            atomicExch(jac_lock, 0);
        }
    }

    // ---------------- adjoint tape ----------------
    __device__ void rec_reset_map()
    {
        for (int i = g.lane; i < 36; i += L) Pm[i] = (i % 7 == 0) ? 1.0 : 0.0;
        g.sync();
    }
    // recording only with a tape; the recording code out of line
    __device__ __forceinline__ void rec_init(double h0)
    {
        if (tape) rec_init_body(h0);
    }
    __device__ __forceinline__ void rec_accept(int q, int qo, const double *l, double inv_xi, double gamma,
                                               double il1, double h, int ncf, int nef)
    {
        if (tape) rec_accept_body(q, qo, l, inv_xi, gamma, il1, h, ncf, nef);
    }
    __device__ __noinline__ void rec_init_body(double h0)
    {
        const double *z0 = V(V_Z0);
        for (int i = g.lane; i < N; i += L) tape[8 + i] = z0[i];
        if (g.lane == 0) { tape[0] = 0.0; tape[1] = h0; tape[2] = 0.0; }
        rec_count = 0;
        rec_reset_map();
    }
    // one accepted step: y_n (= z0 after the correction), the map, the
    // update vector (with the terms of an order increase), gamma, 1/l_1, and
    // the step size and failed attempts of the step
    __device__ __noinline__ void rec_accept_body(int q, int qo, const double *l, double inv_xi, double gamma,
                                                 double il1, double h, int ncf, int nef)
    {
        if (rec_count >= tape_cap) {
            if (g.lane == 0) tape[2] = 1.0;
            return;
        }
        double *r = tape + tape_header(N) + (size_t)rec_count * tape_record(N);
        const double *z0 = V(V_Z0);
        for (int i = g.lane; i < N; i += L) r[i] = z0[i];
        for (int i = g.lane; i < 36; i += L) r[N + i] = Pm[i];
        if (g.lane == 0) {
            double c[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                c[j] = (j <= q) ? l[j] : 0.0;
                if (qo == q + 1 && j >= 1 && j <= q + 1) c[j] += l[j - 1] * inv_xi;
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) r[N + 36 + j] = c[j];
            r[N + 42] = gamma;
            r[N + 43] = il1;
            r[N + 44] = (double)q;
            r[N + 45] = (double)qo;
            r[N + 46] = h;
            r[N + 47] = (double)ncf;
            r[N + 48] = (double)nef;
            tape[0] = (double)(rec_count + 1);
        }
        ++rec_count;
        g.sync();
        rec_reset_map();
    }

    // ---------------- vector operations (lane-strided over N) ----------------
    __device__ __forceinline__ void load_y(int s)
    {
        double *d = V(s);
        for (int i = g.lane; i < N; i += L) d[i] = yg[i];
        g.sync();
    }
    __device__ __forceinline__ void store_y(int s)
    {
        const double *d = V(s);
        for (int i = g.lane; i < N; i += L) yg[i] = d[i];
    }
    __device__ __forceinline__ bool all_finite(int s) const
    {
        const double *d = V(s);
        int bad = 0;
        for (int i = g.lane; i < N; i += L) bad |= !(fabs(d[i]) <= 1.7e308);
        return __all_sync(g.mask, bad == 0);
    }
    __device__ __forceinline__ void set_weights(int s, double rtol)
    {
        const double *y = V(s);
        double *w = V(V_W);
        for (int i = g.lane; i < N; i += L) w[i] = rcp(rtol * fabs(y[i]) + tb.atol[i]);
        g.sync();
    }
    __device__ __forceinline__ double wrms2(int s) const
    {
        const double *a = V(s), *w = V(V_W);
        double acc = 0.0;
        for (int i = g.lane; i < N; i += L) { const double t = a[i] * w[i]; acc += t * t; }
        return g.sum(acc) * invN;
    }
    __device__ __forceinline__ double wrms2_lin(double ca, int sa, double cb, int sb) const
    {
        const double *a = V(sa), *b = V(sb), *w = V(V_W);
        double acc = 0.0;
        for (int i = g.lane; i < N; i += L) {
            const double t = (ca * a[i] + cb * b[i]) * w[i];
            acc += t * t;
        }
        return g.sum(acc) * invN;
    }
    __device__ __forceinline__ void axpby(int o, double ca, int sa, double cb, int sb)
    {
        double *d = V(o);
        const double *a = V(sa), *b = V(sb);
        for (int i = g.lane; i < N; i += L) d[i] = ca * a[i] + cb * b[i];
        g.sync();
    }
    __device__ __forceinline__ void scale(int o, double ca, int sa)
    {
        double *d = V(o);
        const double *a = V(sa);
        for (int i = g.lane; i < N; i += L) d[i] = ca * a[i];
        g.sync();
    }
    // Each lane owns the same elements in every column, so the Nordsieck
    // updates need no synchronisation between columns.
    __device__ __forceinline__ void predict(int q)
    {
        for (int i = g.lane; i < N; i += L) {
            double z[QMAX + 1];
#pragma unroll
            for (int j = 0; j <= QMAX; ++j) z[j] = (j <= q) ? vec[j * NP + i] : 0.0;
#pragma unroll
            for (int k = 0; k < QMAX; ++k)
#pragma unroll
                for (int j = QMAX; j >= 1; --j)
                    if (k < q && j > k && j <= q) z[j - 1] += z[j];
#pragma unroll
            for (int j = 0; j <= QMAX; ++j) if (j <= q) vec[j * NP + i] = z[j];
        }
        g.sync();
    }
    __device__ __forceinline__ void unpredict(int q)
    {
        for (int i = g.lane; i < N; i += L) {
            double z[QMAX + 1];
#pragma unroll
            for (int j = 0; j <= QMAX; ++j) z[j] = (j <= q) ? vec[j * NP + i] : 0.0;
#pragma unroll
            for (int k = QMAX - 1; k >= 0; --k)
#pragma unroll
                for (int j = 1; j <= QMAX; ++j)
                    if (k < q && j > k && j <= q) z[j - 1] -= z[j];
#pragma unroll
            for (int j = 0; j <= QMAX; ++j) if (j <= q) vec[j * NP + i] = z[j];
        }
        g.sync();
    }
    __device__ __forceinline__ void rescale(int q, double eta)
    {
        double f[QMAX + 1];
        f[0] = 1.0;
#pragma unroll
        for (int j = 1; j <= QMAX; ++j) f[j] = f[j - 1] * eta;
        for (int i = g.lane; i < N; i += L) {
#pragma unroll
            for (int j = 1; j <= QMAX; ++j) if (j <= q) vec[j * NP + i] *= f[j];
        }
        if (tape)
            for (int i = g.lane; i < 6; i += L) {
#pragma unroll
                for (int j = 1; j <= QMAX; ++j) if (j <= q) Pm[j * 6 + i] *= f[j];
            }
        g.sync();
    }
    __device__ __forceinline__ void correct(int q, const double *l)
    {
        const double *ac = V(V_ACOR);
        for (int i = g.lane; i < N; i += L) {
            const double a = ac[i];
#pragma unroll
            for (int j = 0; j <= QMAX; ++j) if (j <= q) vec[j * NP + i] += l[j] * a;
        }
        g.sync();
    }
    __device__ __forceinline__ void order_increase(int q, const double *l, double inv_xi)
    {
        const double *ac = V(V_ACOR);
        for (int i = g.lane; i < N; i += L) {
            const double a = ac[i];
            vec[(q + 1) * NP + i] = 0.0;
#pragma unroll
            for (int j = 1; j <= QMAX; ++j)
                if (j <= q + 1) vec[j * NP + i] += l[j - 1] * inv_xi * a;
        }
        g.sync();
    }
    __device__ __forceinline__ void order_decrease(int q, const double *e)
    {
        for (int i = g.lane; i < N; i += L) {
            const double zq = vec[q * NP + i];
#pragma unroll
            for (int j = 1; j < QMAX; ++j) if (j < q) vec[j * NP + i] -= e[j - 1] * zq;
            vec[q * NP + i] = 0.0;
        }
        if (tape)
            for (int i = g.lane; i < 6; i += L) {
                const double pq = Pm[q * 6 + i];
#pragma unroll
                for (int j = 1; j < QMAX; ++j) if (j < q) Pm[j * 6 + i] -= e[j - 1] * pq;
                Pm[q * 6 + i] = 0.0;
            }
        g.sync();
    }
    __device__ __forceinline__ void restart(double h)
    {
        const double *f = V(V_F);
        for (int i = g.lane; i < N; i += L) {
            vec[NP + i] = h * f[i];
#pragma unroll
            for (int j = 2; j <= QMAX; ++j) vec[j * NP + i] = 0.0;
        }
        g.sync();
    }
    __device__ __forceinline__ void newton_init()
    {
        double *ac = V(V_ACOR), *y = V(V_Y);
        const double *z0 = V(V_Z0);
        for (int i = g.lane; i < N; i += L) { ac[i] = 0.0; y[i] = z0[i]; }
        g.sync();
    }
    __device__ __forceinline__ void newton_residual(double h, double il1)
    {
        double *d = V(V_DEL);
        const double *f = V(V_F), *z1 = V(V_Z1), *ac = V(V_ACOR);
        for (int i = g.lane; i < N; i += L) d[i] = (h * f[i] - z1[i]) * il1 - ac[i];
        g.sync();
    }
    __device__ __forceinline__ double newton_update(double c)
    {
        double *d = V(V_DEL), *ac = V(V_ACOR), *y = V(V_Y);
        const double *z0 = V(V_Z0), *w = V(V_W);
        double acc = 0.0;
        for (int i = g.lane; i < N; i += L) {
            const double di = d[i] * c;
            const double a = ac[i] + di;
            ac[i] = a;
            y[i] = z0[i] + a;
            const double t = di * w[i];
            acc += t * t;
        }
        acc = g.sum(acc) * invN;
        g.sync();
        return acc;
    }

    // ---------------- right-hand side (+ Newton matrix) ----------------
    // f(y) of slot sin into slot sout; with jac also M = I - gamma J(y) (or
    // -gamma J without the identity) into mat.  jac is uniform over the
    // group; groups of a warp with and without it share the f part.
    __device__ __forceinline__ int eval(int sin, int sout, double gamma, bool jac, bool add_identity = true)
    {
        return eval_p(V(sin), V(sout), gamma, jac, add_identity);
    }
    __device__ int eval_p(const double *y, double *f, double gamma, bool jac, bool add_identity = true)
    {
        const double T = y[K];
        const double lnT = flog(T), invT = rcp(T);
        double s = 0.0;
        for (int k = g.lane; k < K; k += L) s += y[k] * tb.invW[k];
        s = g.sum(s);
        const double rts = RU * T * s;
        const double rho = P * rcp(rts);
        const double rrho = rts * invP;
        {
            // distinct shared-memory arrays: restrict lets loads of the next
            // species move above this species' stores
            const double *__restrict__ yr = y;
            const double *__restrict__ cpc = tb.cpc, *__restrict__ hc = tb.hc, *__restrict__ sc = tb.sc;
            const double *__restrict__ iW = tb.invW, *__restrict__ xt = tb.exptab;
            double *__restrict__ Cw = C, *__restrict__ Dw = D, *__restrict__ Ew = egi;
            double *__restrict__ Hw = hRT, *__restrict__ Pw = cpR;
            for (int k = g.lane; k < K; k += L) {
                const double *a = cpc + 5 * k, *hh = hc + 6 * k, *ss = sc + 6 * k;
                const double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
                const double hrt = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
                const double sr = ss[0] * lnT + T * (ss[1] + T * (ss[2] + T * (ss[3] + T * ss[4]))) + ss[5];
                const double e = fexp(hrt - sr, xt);
                const double ck = rho * yr[k] * iW[k];
                Cw[k] = ck;
                Dw[k] = e * ck;
                Ew[k] = rcp(e);
                Hw[k] = hrt;
                Pw[k] = cp;
            }
        }
        g.sync();
        const double rtp = RU * T * (1.0 / PATM), irtp = rcp(rtp);
        const double pw[5] = {irtp * irtp, irtp, 1.0, rtp, rtp * rtp};
        const double *__restrict__ Cr = C, *__restrict__ Dr = D, *__restrict__ Er = egi, *__restrict__ Hr = hRT;
        const double *__restrict__ rpar = tb.rpar, *__restrict__ xt = tb.exptab;
        const uint32_t *__restrict__ ridx = tb.ridx;
        double *__restrict__ qw = q, *__restrict__ dTw = dqdT, *__restrict__ uw = uq;
        MT *__restrict__ dqw = dq;
        for (int j = g.lane; j < M; j += L) {
            const uint32_t a = ridx[2 * j], b = ridx[2 * j + 1];
            const int r0 = a & 0xff, r1 = (a >> 8) & 0xff, r2 = (a >> 16) & 0xff, p0 = a >> 24;
            const int p1 = b & 0xff, p2 = (b >> 8) & 0xff, dnu = (int)((b >> 16) & 0xff) - 8;
            const double *rp = rpar + 3 * j;
            const double kf = fexp(rp[0] + rp[1] * lnT - rp[2] * invT, xt);
            // kr prod_p C_p = kf / Kc prod_p C_p = kf * G * B with
            // G = prod_r exp(-g_r) (P_atm/RT)^-dnu and B = prod_p exp(g_p) C_p
            const double c0 = Cr[r0], c1 = Cr[r1], c2 = Cr[r2];
            const double A = c0 * c1 * c2;
            const double G = (Er[r0] * Er[r1] * Er[r2]) * pw[dnu + 2];
            const double B = Dr[p0] * Dr[p1] * Dr[p2];
            qw[j] = kf * (A - G * B);
            if (jac) {
                MT *dj = dqw + 6 * j;
                const double rkf = kf * G;                 // kr = rkf prod_p exp(g_p)
                const double fwd = kf * A, rev = rkf * B;
                const double gkf = gamma * kf, grk = gamma * rkf;
                const double D0 = Dr[p0], D1 = Dr[p1], D2 = Dr[p2];
                dj[0] = (MT)(gkf * (c1 * c2));
                dj[1] = (MT)(gkf * (c0 * c2));
                dj[2] = (MT)(gkf * (c0 * c1));
                // gamma kr prod_{p != i} C_p = gamma rkf exp(g_i) prod_{p != i} D_p
                dj[3] = (MT)(-grk * rcp(Er[p0]) * (D1 * D2));
                dj[4] = (MT)(-grk * rcp(Er[p1]) * (D0 * D2));
                dj[5] = (MT)(-grk * rcp(Er[p2]) * (D0 * D1));
                const double af = rp[1] + rp[2] * invT;
                const double dH = (Hr[p0] + Hr[p1] + Hr[p2]) - (Hr[r0] + Hr[r1] + Hr[r2]);
                dTw[j] = gamma * invT * (af * fwd - (af - dH + (double)dnu) * rev);
                // sum_m C_m dq_j/dC_m = n_r fwd - n_p rev (each product term is
                // homogeneous in C): formed in FP64 here, because summing the
                // large, nearly cancelling row entries instead loses it in FP32
                const int nr = (int)(b >> 24), np = nr + dnu;
                uw[j] = gamma * ((double)nr * fwd - (double)np * rev);
            }
        }
        g.sync();
        double hw = 0.0, cpm = 0.0;
        {
            const double *__restrict__ qr = q, *__restrict__ nu = tb.inc_nu, *__restrict__ Hr2 = hRT;
            const double *__restrict__ Pr = cpR, *__restrict__ yr = y, *__restrict__ Wr = tb.W, *__restrict__ iW = tb.invW;
            const int32_t *__restrict__ ip = tb.inc_ptr, *__restrict__ ij = tb.inc_j;
            double *__restrict__ fw = f, *__restrict__ ww = wdot;
            for (int k = g.lane; k < K; k += L) {
                double wd = 0.0;
                const int e1 = ip[k + 1];
                for (int e = ip[k]; e < e1; ++e) wd += nu[e] * qr[ij[e]];
                fw[k] = wd * Wr[k] * rrho;
                hw += Hr2[k] * wd;
                cpm += yr[k] * Pr[k] * iW[k];
                if (jac) ww[k] = wd;
            }
        }
        hw = g.sum(hw);
        cpm = g.sum(cpm);
        const double fT = -T * hw * rcp(rho * cpm);
        if (g.lane == 0) f[K] = fT;
        last_rho = rho;
        last_cpm = cpm;
        last_T = T;
        g.sync();
        if (!jac) return 1;

        // ---- Newton matrix M = I - gamma J (gamma folded into dq, dqdT) ----
        // rows k < K of gamma*Jc (in MT), and gamma * dwdot/dT, gamma * u (in FP64)
        {
            const MT *nu = tb.template nu<MT>();
            for (int k = g.lane; k < K; k += L) {
                MT *row = mat + k * N;
                for (int m = 0; m < N; ++m) row[m] = (MT)0;
                double wt = 0.0, uk = 0.0;
                const int e1 = tb.inc_ptr[k + 1];
                for (int e = tb.inc_ptr[k]; e < e1; ++e) {
                    const int j = tb.inc_j[e];
                    const MT n = nu[e];
                    const double nd = tb.inc_nu[e];
                    const uint32_t a = tb.ridx[2 * j], b = tb.ridx[2 * j + 1];
                    const MT *dj = dq + 6 * j;
                    wt += nd * dqdT[j];
                    uk += nd * uq[j];
                    row[a & 0xff] += n * dj[0];
                    row[(a >> 8) & 0xff] += n * dj[1];
                    row[(a >> 16) & 0xff] += n * dj[2];
                    row[a >> 24] += n * dj[3];
                    row[b & 0xff] += n * dj[4];
                    row[(b >> 8) & 0xff] += n * dj[5];
                }
                wT[k] = wt;
                u[k] = uk;
            }
        }
        g.sync();
        // scalars of the temperature row
        double sU = 0.0, sA1 = 0.0, sA2 = 0.0, sA3 = 0.0;
        for (int k = g.lane; k < K; k += L) {
            sU += hRT[k] * u[k];
            sA1 += cpR[k] * wdot[k];
            sA2 += hRT[k] * (wT[k] - u[k] * invT);
            const double *dc = tb.dcp + 4 * k;
            sA3 += y[k] * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3]))) * tb.invW[k];
        }
        sU = g.sum(sU); sA1 = g.sum(sA1); sA2 = g.sum(sA2); sA3 = g.sum(sA3);
        const double Wbar = rcp(s);
        const double icpm = rcp(cpm);
        const double rtP = RU * T * invP;               // Wbar / rho
        // temperature row (from the unscaled-by-W rows of gamma*Jc)
        for (int l = g.lane; l < K; l += L) {
            MT Sl = (MT)0;
            for (int k = 0; k < K; ++k) Sl += (MT)hRT[k] * mat[k * N + l];
            const double gJ = -(tb.invW[l] * icpm) *
                              (T * ((double)Sl - rtP * sU) + gamma * fT * (cpR[l] - cpm * Wbar));
            xs[l] = (MT)gJ;   // staged: row K is written after the k-rows are done
        }
        const double gJTT = -(gamma * sA1 + T * sA2) * rcp(rho * cpm) - gamma * fT * (-invT + sA3 * icpm);
        g.sync();
        // species rows: gamma*J_kl = (W_k/W_l)(gamma Jc_kl + (Ru T/P) gamma (wdot_k - u_k)), then M = I - gamma J
        {
            const MT *iw = tb.template iw<MT>();
            for (int k = g.lane; k < K; k += L) {
                MT *row = mat + k * N;
                const MT ck = (MT)(rtP * (gamma * wdot[k] - u[k]));
                const MT Wk = (MT)tb.W[k];
                for (int l = 0; l < K; ++l) {
                    const MT gJ = (Wk * iw[l]) * (row[l] + ck);
                    row[l] = ((l == k && add_identity) ? (MT)1 : (MT)0) - gJ;
                }
                row[K] = (MT)(-(tb.W[k] * rrho) * (wT[k] + (gamma * wdot[k] - u[k]) * invT));
            }
        }
        for (int l = g.lane; l < K; l += L) mat[K * N + l] = -xs[l];
        if (g.lane == 0) mat[K * N + K] = (MT)((add_identity ? 1.0 : 0.0) - gJTT);
        g.sync();
        return 1;
    }

    __device__ __forceinline__ void rhs(int a, int b) { eval(a, b, 0.0, false); }
    // the starting step's f evaluations (once per cell): out of line, so
    // that the kernel's hot loop does not carry two more copies of eval
    __device__ __noinline__ void rhs_start(int a, int b) { eval(a, b, 0.0, false); }
    // The f evaluation of a Newton iteration, f(y) into V_F; with setup also
    // the Newton matrix at y, factored (0: singular).  One call site for
    // both, so groups of a warp that set up and groups that do not share
    // the right-hand-side work.
    __device__ __forceinline__ int newton_f(bool setup, double gamma)
    {
        if (setup && jac_dq) {
            eval(V_Y, V_F, gamma, false);
            setup_dq(gamma);
            release_setup();
            return factor();
        }
        eval(V_Y, V_F, gamma, setup);
        if (!setup) return 1;
        release_setup();                 // the matrix is assembled: scratch free
        return factor();
    }
    // right-hand sides a matrix build costs on top of the Newton iteration's
    __device__ __forceinline__ int f_per_setup() const { return jac_dq ? N : 0; }

    // M = I - gamma J with J by forward difference quotients (solution
    // approaches 3A/3B of Table 1, Sec. 4.1.4): column j from
    // f(y + inc e_j), inc = max(sqrt(eps) |y_j|, sqrt(eps) / w_j) rounded to
    // the representable step; f(y) is the Newton iteration's (in V_F).  The
    // perturbed f goes to the Newton-matrix scratch, which a difference-
    // quotient build does not otherwise need.  Out of line: N right-hand
    // sides per build.
    __device__ __noinline__ void setup_dq(double gamma)
    {
        double *fp = reinterpret_cast<double *>(dq);
        const double *y = V(V_Y), *f0 = V(V_F), *w = V(V_W);
        double *yp = V(V_DEL);
        const double se = 1.4901161193847656e-08;          // sqrt(DBL_EPSILON) = 2^-26
        for (int j = 0; j < N; ++j) {
            for (int i = g.lane; i < N; i += L) yp[i] = y[i];
            const double yj = y[j];
            const double inc0 = fmax(se * fabs(yj), se / w[j]);
            const double ypj = yj + inc0, inc = ypj - yj;
            g.sync();
            if (g.lane == 0) yp[j] = ypj;
            g.sync();
            eval_p(yp, fp, 0.0, false);
            for (int i = g.lane; i < N; i += L)
                mat[i * N + j] = (MT)((i == j ? 1.0 : 0.0) - gamma * ((fp[i] - f0[i]) / inc));
            g.sync();
        }
    }

    // ---------------- matrix-free linear solver ----------------
    // The inexact Newton iteration's linear solve (solution approaches 1A/1B
    // of Table 1; Eqs. linear and stop_linear, Sec. 2): M x = b for the
    // residual b in V_DEL, M = I - gamma J at the iterate y (V_Y, f(y) in
    // V_F), by GMRES on the system scaled by S = diag(w) (V_W),
    //   (S M S^-1) xt = S b,  x = S^-1 xt,
    // unpreconditioned, with J v by a forward difference along v,
    //   J v = (f(y + sig v) - f(y)) / sig,  sig = 1 / ||v||_wrms.
    // Modified Gram-Schmidt and Givens rotations; stops once the rotated
    // residual |g_{k+1}| (the scaled residual's 2-norm) is at most
    // tol = 0.05 (NLS_COEF / C_q) sqrt(N) -- Eq. stop_linear's c_l = 0.05 of
    // the Newton tolerance, a WRMS bound, in the 2-norm -- or after
    // krylov_dim(N) iterations, and leaves x in V_DEL (0 when ||S b|| <= tol).  Returns the f evaluations it made.  The lanes own the
    // vector elements i = lane (mod L) as everywhere else; lane 0 keeps the
    // Hessenberg matrix and the rotations, and the lanes read the rotated
    // residual back after a group barrier, so the exit is uniform.  Out of
    // line: it only runs when the Krylov solver is selected.
    __device__ __noinline__ int solve_krylov(double gamma, double Cq)
    {
        const double tol = 0.05 * (NLS_COEF / Cq) * sqrt((double)N);
        const int l = krylov_dim(N);
        double *Vb = this->kry, *H = Vb + (l + 1) * N, *cs = H + (l + 1) * l, *sn = cs + l;
        double *gv = sn + l, *cv = gv + (l + 1), *yt = cv + l, *ft = yt + N;
        double *b = V(V_DEL);
        const double *y = V(V_Y), *fy = V(V_F), *w = V(V_W);
        double acc = 0.0;
        for (int i = g.lane; i < N; i += L) {
            const double v = w[i] * b[i];
            Vb[i] = v;
            b[i] = 0.0;
            acc += v * v;
        }
        const double beta = sqrt(g.sum(acc));
        if (!(beta > tol)) { g.sync(); return 0; }
        for (int i = g.lane; i < N; i += L) Vb[i] = Vb[i] / beta;
        if (g.lane == 0) gv[0] = beta;
        int k = 0, nfe = 0;
        for (int j = 0; j < l; ++j) {
            const double *vj = Vb + j * N;
            double *vn = Vb + (j + 1) * N;
            // S M S^-1 v_j: u = S^-1 v_j, sig = 1/||u||_wrms, y + sig u
            double a2 = 0.0;
            for (int i = g.lane; i < N; i += L) {
                const double uw = (vj[i] / w[i]) * w[i];
                a2 += uw * uw;
            }
            const double sig = 1.0 / sqrt(g.sum(a2) * invN);
            for (int i = g.lane; i < N; i += L) yt[i] = y[i] + sig * (vj[i] / w[i]);
            g.sync();
            eval_p(yt, ft, 0.0, false);
            ++nfe;
            for (int i = g.lane; i < N; i += L)
                vn[i] = w[i] * (vj[i] / w[i] - gamma * ((ft[i] - fy[i]) / sig));
            // modified Gram-Schmidt against v_0 .. v_j
            for (int m = 0; m <= j; ++m) {
                const double *vm = Vb + m * N;
                double hp = 0.0;
                for (int i = g.lane; i < N; i += L) hp += vn[i] * vm[i];
                const double h = g.sum(hp);
                for (int i = g.lane; i < N; i += L) vn[i] -= h * vm[i];
                if (g.lane == 0) H[m * l + j] = h;
            }
            double hp = 0.0;
            for (int i = g.lane; i < N; i += L) hp += vn[i] * vn[i];
            const double hn = sqrt(g.sum(hp));
            if (g.lane == 0) {
                // the earlier rotations on column j, then the one that zeroes H[j+1][j]
                for (int m = 0; m < j; ++m) {
                    const double a = H[m * l + j], bb = H[(m + 1) * l + j];
                    H[m * l + j] = cs[m] * a + sn[m] * bb;
                    H[(m + 1) * l + j] = -sn[m] * a + cs[m] * bb;
                }
                const double a = H[j * l + j], r = sqrt(a * a + hn * hn);
                cs[j] = r > 0.0 ? a / r : 1.0;
                sn[j] = r > 0.0 ? hn / r : 0.0;
                H[j * l + j] = r;
                gv[j + 1] = -sn[j] * gv[j];
                gv[j] = cs[j] * gv[j];
            }
            g.sync();
            k = j + 1;
            if (fabs(gv[j + 1]) <= tol || !(hn > 0.0)) break;
            for (int i = g.lane; i < N; i += L) vn[i] = vn[i] / hn;
        }
        // H[0:k][0:k] c = g[0:k] (upper triangular), x = S^-1 sum_m c_m v_m
        if (g.lane == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double s = gv[i];
                for (int m = i + 1; m < k; ++m) s -= H[i * l + m] * cv[m];
                cv[i] = s / H[i * l + i];
            }
        }
        g.sync();
        for (int i = g.lane; i < N; i += L) {
            double xt = 0.0;
            for (int m = 0; m < k; ++m) xt += cv[m] * Vb[m * N + i];
            b[i] = xt / w[i];
        }
        g.sync();
        return nfe;
    }

    __device__ int factor() { return lu_factor<L, MT>(g, mat, N, perm, dinv, nullptr); }
    __device__ void solve(int sb) { lu_solve<L, MT>(g, mat, N, perm, dinv, xs, V(sb)); }
};

}  // namespace sunb
