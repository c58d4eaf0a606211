// Shared definitions of the batched BDF integrator's CUDA path (sm_103a).
//
// Method: arXiv 2405.01713 (Balos et al.), Sec. 2 - every cell's ODE
// y' = f(t, y; p) is advanced by an adaptive-order (1..5), adaptive-step BDF
// method with the WRMS error test (Eq. wrms) and a modified Newton iteration
// stopped by Eq. stop_newton (c_eps = 0.1, c_r = 0.3) on I - gamma J with a
// dense Jacobian and a pivoted LU (Table 1 approach 2A; Sec. 4.1.4, 4.1.6).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace sunb {

// ---------------- logarithm used by the right-hand sides ----------------
// log(x) by table-driven reduction (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990), with 128 table entries:
//   x = 2^m (F + f),  F = 1 + j/128 (the leading 7 mantissa bits),
//   0 <= f < 1/128,  log x = m ln2 + log F + log1p(f/F),
// f exact (Sterbenz), f/F = f * (1/F) from the table, log1p(r) by its
// degree-7 Taylor polynomial (|r| < 1/128: truncation below 2e-18).  ln2 is
// split as LN2_HI (42 significant bits, so m LN2_HI is exact) + LN2_LO, and
// log F as hi + lo in the table.  g_log_tab[j] = 1/F, [128 + j] = log F
// (hi), [256 + j] = log F (lo), filled by the host (fill_math_tables) in
// every translation unit that evaluates it.  Zero, negative, subnormal, infinite
// and NaN x go to the library log.  Error: within 2 ulp of log x, and
// within 4e-16 absolute where log x is small and m != 0 (x just below 1).
// The library functions for the arguments the table methods leave out: out
// of line, so that their code is not repeated at every call site.
static __device__ __noinline__ double log_outside(double x) { return log(x); }
static __device__ __noinline__ double exp_outside(double x) { return exp(x); }

constexpr int LOG_TABLE_SIZE = 128;   // the shift below (>> 13, & 127) assumes 128
static __device__ double g_log_tab[3 * LOG_TABLE_SIZE];

__device__ __forceinline__ double flog(double x)
{
    const int hi = __double2hiint(x);
    if (hi < 0x00100000 || hi >= 0x7ff00000) return log_outside(x);   // not a positive normal number
    const int m = (hi >> 20) - 1023;
    const int j = (hi >> 13) & (LOG_TABLE_SIZE - 1);
    const double xm = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));   // [1, 2)
    const double F = __hiloint2double(0x3ff00000 | (j << 13), 0);                            // 1 + j/128
    const double r = (xm - F) * __ldg(g_log_tab + j);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(r, q, 1.0 / 5.0);
    q = fma(r, q, -0.25);
    q = fma(r, q, 1.0 / 3.0);
    q = fma(r, q, -0.5);
    const double s = (r * r) * q;                                // log1p(r) - r
    const double md = (double)m;
    const double h = fma(md, 0x1.62e42fefa3800p-1, __ldg(g_log_tab + LOG_TABLE_SIZE + j));
    const double l = fma(md, 0x1.ef35793c76730p-45, __ldg(g_log_tab + 2 * LOG_TABLE_SIZE + j));
    return h + (r + (s + l));
}

// ---------------- exponential used by the right-hand sides ----------------
// exp(x) by table-driven range reduction (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989), with 64 table entries:
//   x = (64 m + j) ln2/64 + r,  |r| <= ln2/128,
//   exp(x) = 2^m * 2^(j/64) * (1 + p(r)),
// p(r) the degree-5 Taylor polynomial of e^r - 1 (truncation below 4e-17
// relative).  ln2/64 is split as C1 + C2 with C1 of 32 significant bits, so
// that n C1 is exact; n is the nearest integer to 64 x/ln2, read from the
// low word of x 64/ln2 + 1.5*2^52.  tab[j] = 2^(j/64) rounded to double
// (EXP_TABLE_SIZE entries: a shared-memory copy in the kernels, or
// g_exp_tab, filled by fill_math_tables).  For |x| >= 704, where
// 2^m would leave the normal range, and for NaN the library exp is used.
// Accuracy: within 2 ulp of exp (checked against it by the GPU tests).
constexpr int EXP_TABLE_SIZE = 64;   // the shifts below (>> 6, & 63) assume 64
static __device__ double g_exp_tab[EXP_TABLE_SIZE];
__device__ __forceinline__ double fexp(double x, const double *__restrict__ tab)
{
    if (!(fabs(x) < 704.0)) return exp_outside(x);
    const double shift = 6755399441055744.0;                 // 1.5 * 2^52
    const double t = fma(x, 0x1.71547652b82fep+6, shift);    // 64 / ln 2
    const int n = __double2loint(t);
    const double nd = t - shift;
    double r = fma(-nd, 0x1.62e42ff000000p-7, x);            // C1
    r = fma(-nd, -0x1.718432a1b0e26p-41, r);                 // C2
    double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    p = fma(r, p, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r, p, 1.0);
    p *= r;
    const double tj = tab[n & (EXP_TABLE_SIZE - 1)];
    const double v = fma(tj, p, tj);
    return __hiloint2double(__double2hiint(v) + ((n >> 6) << 20), __double2loint(v));
}


constexpr int QMAX = 5;
constexpr int NVEC = 12;            // per-cell vectors held by the controller

// physical constants (CODATA values; cgs units, Ea in cal/mol)
constexpr double RU = 8.314462618e7;
constexpr double RC = 1.98720425864083;
constexpr double PATM = 1013250.0;
constexpr double LN1E4 = 9.210340371976184;

// Step-control constants.  The paper fixes c_eps = 0.1 and c_r = 0.3
// (Eq. stop_newton); the rest are readings of points it leaves open:
// growth limits, failure factors, biases and the rebuild policy.
constexpr double NLS_COEF = 0.1;       // c_eps
constexpr double CRDOWN = 0.3;         // c_r
constexpr double RDIV = 2.0;           // divergence ratio of successive corrections
constexpr int MAXCOR = 3;              // Newton iterations per attempt
constexpr int MXNEF = 7;               // error-test failures per step
constexpr int MXNEF1 = 3;              // failures before the order-1 restart
constexpr int MXNCF = 10;              // Newton failures per step
constexpr int MSBP = 20;               // steps between matrix rebuilds
constexpr double DGMAX = 0.3;          // |gamma/gamma_M - 1| that forces a rebuild
constexpr double ETA_CF = 0.25;        // step factor after a Newton failure
constexpr double ETA_MIN_EF = 0.1;     // error-test failure factor bounds
constexpr double ETA_MAX_EF = 0.9;
constexpr double ETA_THRESH = 1.5;     // below this the step is kept
constexpr double ETA_MAX_FIRST = 1e4;  // growth cap after the first step
constexpr double ETA_MAX = 10.0;       // growth cap afterwards
constexpr float BIAS_QM1 = 6.0f, BIAS_Q = 6.0f, BIAS_QP1 = 10.0f;   // (single precision: eta_from)

enum Status : int32_t {
    ST_SUCCESS = 0, ST_TOO_MUCH_WORK = -1, ST_ERR_FAILURE = -3,
    ST_CONV_FAILURE = -4, ST_H_TOO_SMALL = -5, ST_NONFINITE = -6
};

// per-cell counters, in the order of the public [C, 8] statistics array
struct CellStats {
    int32_t nst, nfe, nje, nni, ncf, nef, qlast, status;
};

// Integration controls shared by every cell of a launch.
struct Controls {
    double rtol;
    double t0, tout;
    int32_t max_steps;
    int32_t max_order;
};

// Vector slots of the controller.
enum Vec : int {
    V_Z0 = 0, V_Z1 = 1,  // Nordsieck columns 0..5 occupy slots 0..5
    V_ACOR = 6, V_Y = 7, V_F = 8, V_W = 9, V_DEL = 10, V_KS = 11
};

__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// ---------------- host side of the math tables ----------------
// 2^(j/64) rounded to double: the table of fexp.
static inline void exp_table_values(double *t)
{
    for (int j = 0; j < EXP_TABLE_SIZE; ++j) t[j] = (double)exp2l((long double)j / (long double)EXP_TABLE_SIZE);
}

// This translation unit's g_exp_tab and g_log_tab on the current device
// (1/F and log F in two parts for F = 1 + j/128).  Returns cudaSuccess or
// the copy's error.
static inline cudaError_t fill_math_tables()
{
    double e[EXP_TABLE_SIZE];
    exp_table_values(e);
    double t[3 * LOG_TABLE_SIZE];
    for (int j = 0; j < LOG_TABLE_SIZE; ++j) {
        const long double F = 1.0L + (long double)j / (long double)LOG_TABLE_SIZE;
        const long double lf = logl(F);
        t[j] = (double)(1.0L / F);
        t[LOG_TABLE_SIZE + j] = (double)lf;
        t[2 * LOG_TABLE_SIZE + j] = (double)(lf - (long double)t[LOG_TABLE_SIZE + j]);
    }
    const cudaError_t a = cudaMemcpyToSymbol(g_exp_tab, e, sizeof(e));
    const cudaError_t b = cudaMemcpyToSymbol(g_log_tab, t, sizeof(t));
    return a != cudaSuccess ? a : b;
}

// Header and record sizes (doubles) of a cell's tape: the header is
// [count, h0, overflow, 5 spare, y0 (N)]; a record is y_n (N), the column
// map P (6 x 6, row = output column), the update vector c (6), gamma, 1/l_1,
// q, q_out, then the step's control decisions: its size h_n and the Newton
// and error-test failures of its attempts (ncf, nef).
__host__ __device__ __forceinline__ int tape_header(int N) { return 8 + N; }
__host__ __device__ __forceinline__ int tape_record(int N) { return N + 49; }

}  // namespace sunb
