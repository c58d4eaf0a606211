/* CPU oracle for the batched BDF integrator: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 implementation of what the CUDA path computes, one cell
 * at a time, used by the tests, by smoke() and by the benchmark's CPU
 * baseline leg.  No product code path may include, link or call it, and it
 * shares no code with the CUDA library.
 *
 * Every function cites the passage of arXiv 2405.01713 (Balos et al.,
 * "SUNDIALS Time Integrators for Exascale Applications with Many Independent
 * ODE Systems") that it follows; where the paper is silent, the comment
 * states the reading taken.
 */
#ifndef SUNB_ORACLE_H
#define SUNB_ORACLE_H

#include <stdint.h>

#define ORC_RU 8.314462618e7      /* gas constant, erg/(mol K) */
#define ORC_RC 1.98720425864083   /* gas constant, cal/(mol K) */
#define ORC_PATM 1013250.0        /* standard pressure, dyn/cm^2 */
#define ORC_LN1E4 9.210340371976184 /* ln(1e4) */

enum { ORC_ROBERTSON = 0, ORC_MECHANISM = 1, ORC_COSMOLOGY = 2, ORC_LINEAR = 3 };

enum {
    ORC_SUCCESS = 0, ORC_TOO_MUCH_WORK = -1, ORC_ERR_FAILURE = -3,
    ORC_CONV_FAILURE = -4, ORC_H_TOO_SMALL = -5, ORC_NONFINITE = -6
};

typedef struct {
    int kind;            /* ORC_ROBERTSON | ORC_MECHANISM | ORC_COSMOLOGY | ORC_LINEAR */
    int n;               /* unknowns per cell */
    int nparams;         /* per-cell parameters (row length of params) */
    const double *params;/* [ncells, nparams] */
    /* mechanism tables */
    int K, M;
    const double *W, *nasa, *lnA, *beta, *Ea;
    const int32_t *react, *prod;
    /* cooling table */
    int nknots;
    const double *lnT, *lnLam;
    double gamma_heat;
} orc_problem;

typedef struct {
    double rtol;
    const double *atol;  /* [n] */
    int max_steps;
    int max_order;       /* 1..5 */
    int jac_mode;        /* 0: complex step, 1: forward difference */
    int lin_solver;      /* 0: dense LU (modified Newton), 1: GMRES (inexact Newton) */
    int method;          /* 0: BDF (CVODE kind), 1: explicit Runge-Kutta 4(3) (ARKODE kind) */
} orc_options;

/* per-cell counters, in this order */
typedef struct {
    int32_t nst, nfe, nje, nni, ncf, nef, qlast, status;
} orc_stats;

#endif
