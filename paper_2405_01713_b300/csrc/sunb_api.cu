// Host side of the C ABI declared in include/sunb.h, and the kernels it
// launches.  One process, one GPU, one stream per context; all workspace is
// allocated in sunb_create (the paper's Sec. 4.3.1 measures how much
// per-step allocation costs), except the staging buffer of
// sunb_integrate_host, allocated on its first use.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sunb.h"
#include "sunb_common.cuh"
#include "bdf_control.cuh"
#include "cell_thread.cuh"
#include "cell_group.cuh"
#include "kernels_thread.cuh"

using namespace sunb;

// ============================================================ device side

struct MechArgs {
    const unsigned char *tab;
    MechTabOffsets off;
    CellLayout lay;
    int cells_per_cta;
    int schedule;
    double invN;
    Controls ctl;
    long long n_mech;
    double *y_mech;
    const double *p_mech;
    int32_t *stats_mech, *status_mech;
    unsigned long long *queue;   // [0] mechanism cells, [1] cosmology cells
    // cosmology cells of a mixed launch
    long long n_cosmo;
    double *y_cosmo;
    const double *p_cosmo;
    int32_t *stats_cosmo, *status_cosmo;
    CoolArgs cool;
    double atol_cosmo;
    int cool_smem_off;
    // discrete-adjoint tape (null: not recorded)
    double *tape;
    long long tape_stride;
    int tape_cap;
    // Newton-matrix scratch shared per warp (mech_kernel; dq_off < 0: in the cell)
    int dq_off, dq_bytes, lock_off;
    int jac_dq;                  // 1: difference-quotient Newton matrix
    // GMRES scratch, kry_stride doubles per lane group (null: direct solves)
    double *kry;
    int kry_stride;
};

template <int L>
__device__ __forceinline__ unsigned group_mask()
{
    if constexpr (L == 32) {
        return 0xffffffffu;
    } else {
        const int w = threadIdx.x & 31;
        return ((1u << L) - 1u) << (w & ~(L - 1));
    }
}

// Persistent mechanism kernel: L lanes per cell, cells_per_cta cells per
// CTA, one CTA set per SM.  In a mixed launch the mechanism cells (the
// larger ones) go first; threads whose group finds the mechanism queue
// empty fill the kernel's tail with cosmology cells, one per thread.
// Counters: queue[0] mechanism cells handed out, queue[1] cosmology cells
// handed out, queue[2] mechanism cells finished (mixed launches).
template <int L, typename MT, bool COSMO, bool KRY>
__global__ void __launch_bounds__(256) mech_kernel(const MechArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    stage_bytes(smem, a.tab, a.off.bytes);
    CoolingSmem cool;
    if (COSMO) cool = stage_cooling(smem + a.cool_smem_off, a.cool);
    int *locks = reinterpret_cast<int *>(smem + a.lock_off);
    if (a.dq_off >= 0)
        for (int i = threadIdx.x; i < (int)(blockDim.x + 31) / 32; i += blockDim.x) locks[i] = 0;
    __syncthreads();

    const int gid = threadIdx.x / L;
    GroupCell<L, MT, KRY> c;
    c.g.lane = threadIdx.x % L;
    c.g.mask = group_mask<L>();
    c.tb = mech_tab_at(smem, a.off);
    c.N = a.off.N; c.K = a.off.K; c.M = a.off.M;
    c.invN = a.invN;
    c.bind(smem + a.off.bytes + gid * a.lay.bytes, a.lay);
    if (a.dq_off >= 0) {   // one Newton-matrix scratch per warp, locked when groups share it
        const int w = threadIdx.x >> 5;
        c.set_jac_scratch(smem + a.dq_off + w * a.dq_bytes, L < 32 ? locks + w : nullptr);
    }
    c.jac_dq = a.jac_dq != 0;
    if constexpr (KRY) c.kry = a.kry + ((long long)blockIdx.x * a.cells_per_cta + gid) * a.kry_stride;

    const unsigned wmask = launched_warp_mask();
    long long next = (long long)blockIdx.x * a.cells_per_cta + gid;
    const long long stride = (long long)gridDim.x * a.cells_per_cta;
    run_cells(
        c, a.ctl, wmask,
        [&]() -> long long {
            long long cell;
            if (a.schedule == SUNB_SCHED_QUEUE) cell = grab_group(a.queue, c.g.lane, c.g.mask, L);
            else { cell = next; next += stride; }
            return cell < a.n_mech ? cell : -1;
        },
        [&](long long cell) {
            c.P = a.p_mech[cell];
            c.invP = rcp(c.P);
            c.yg = a.y_mech + cell * c.N;
            c.tape = a.tape ? a.tape + cell * a.tape_stride : nullptr;
            c.tape_cap = a.tape_cap;
        },
        [&](long long cell, const CellStats &st) {
            if (c.g.lane == 0) {
                write_stats(a.stats_mech, a.status_mech, cell, st);
                if (COSMO) atomicAdd(a.queue + 2, 1ull);
            }
        });
    if (COSMO) {
        // While other groups still integrate mechanism cells, idle threads
        // take cosmology cells (one per thread) from the shared counter;
        // once every mechanism cell is done they stop, and the cosmology
        // kernel that follows on the stream runs the rest at full occupancy.
        __syncwarp(wmask);
        ThreadCell<CosmologyProblem> tc;
        tc.prob.tab = &cool;
        tc.atol[0] = a.atol_cosmo;
        run_cells(
            tc, a.ctl, wmask,
            [&]() -> long long {
                if (*reinterpret_cast<volatile unsigned long long *>(a.queue + 2) >=
                    (unsigned long long)a.n_mech)
                    return -1;
                const long long cell = grab_thread(a.queue + 1);
                return cell < a.n_cosmo ? cell : -1;
            },
            [&](long long cell) {
                tc.prob.load(a.p_cosmo, cell);
                tc.yg = a.y_cosmo + cell;
            },
            [&](long long cell, const CellStats &st) {
                write_stats(a.stats_cosmo, a.status_cosmo, cell, st);
            });
    }
}

// Batched right-hand side (mode 0) or Jacobian (mode 1) of a mechanism:
// one warp per cell, results to out ([n, N] or [n, N, N]).
__global__ void __launch_bounds__(128) mech_eval_kernel(const MechArgs a, const double *y,
                                                        double *out, long long n, int mode)
{
    extern __shared__ __align__(16) unsigned char smem[];
    stage_bytes(smem, a.tab, a.off.bytes);
    __syncthreads();
    const int gid = threadIdx.x / 32;
    GroupCell<32, double> c;
    c.g.lane = threadIdx.x % 32;
    c.g.mask = 0xffffffffu;
    c.tb = mech_tab_at(smem, a.off);
    c.N = a.off.N; c.K = a.off.K; c.M = a.off.M;
    c.invN = a.invN;
    c.bind(smem + a.off.bytes + gid * a.lay.bytes, a.lay);
    const int N = c.N;
    for (long long cell = (long long)blockIdx.x * a.cells_per_cta + gid; cell < n;
         cell += (long long)gridDim.x * a.cells_per_cta) {
        c.P = a.p_mech[cell];
        c.invP = rcp(c.P);
        c.yg = const_cast<double *>(y) + cell * N;
        c.load_y(V_Y);
        if (mode == 0) {
            c.rhs(V_Y, V_F);
            for (int i = c.g.lane; i < N; i += 32) out[cell * N + i] = c.V(V_F)[i];
        } else {
            c.eval(V_Y, V_F, -1.0, true, false);
            for (int i = c.g.lane; i < N * N; i += 32) out[cell * N * N + i] = (double)c.mat[i];
        }
        c.g.sync();
    }
}

template <class Prob>
__global__ void thread_eval_kernel(const ThreadArgs a, const double *y, double *out, long long n, int mode)
{
    __shared__ __align__(16) double cool_s[3 * 256 + EXP_TABLE_SIZE + 128];
    CoolingSmem cool;
    if (Prob::N == 1) cool = stage_cooling(reinterpret_cast<unsigned char *>(cool_s), a.cool);
    __syncthreads();
    constexpr int N = Prob::N;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        Prob p;
        if constexpr (N == 1) p.tab = &cool;
        p.load(a.params, cell);
        double yy[N], f[N], J[N][N];
        for (int i = 0; i < N; ++i) yy[i] = y[cell * N + i];
        if (mode == 0) {
            p.rhs(yy, f);
            for (int i = 0; i < N; ++i) out[cell * N + i] = f[i];
        } else {
            p.jac(yy, J);
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) out[(cell * N + i) * N + j] = J[i][j];
        }
    }
}

// Batched LU factor + solve: one warp per system, matrix staged in shared memory.
template <typename MT>
__global__ void __launch_bounds__(128) lu_batched_kernel(int n, long long batch, MT *A, int32_t *piv,
                                                         MT *b, int32_t *info, int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x / 32;
    unsigned char *base = smem + w * per_warp_bytes;
    MT *mat = reinterpret_cast<MT *>(base);
    MT *dinv = mat + n * n;
    MT *xs = dinv + n;
    int32_t *perm = reinterpret_cast<int32_t *>(xs + n);
    int32_t *pv = perm + n;
    Grp<32> g;
    g.lane = threadIdx.x % 32;
    g.mask = 0xffffffffu;
    for (long long s = (long long)blockIdx.x * (blockDim.x / 32) + w; s < batch;
         s += (long long)gridDim.x * (blockDim.x / 32)) {
        MT *As = A + s * n * n;
        for (int i = g.lane; i < n * n; i += 32) mat[i] = As[i];
        g.sync();
        const int ok = lu_factor<32, MT>(g, mat, n, perm, dinv, pv);
        int bad = n;
        if (!ok) {   // first column without a usable pivot
            for (int k = 0; k < n; ++k) {
                if (!(fabs((double)mat[k * n + k]) > 0.0)) { bad = k; break; }
            }
        }
        lu_solve<32, MT, MT>(g, mat, n, perm, dinv, xs, b + s * n);
        for (int i = g.lane; i < n * n; i += 32) As[i] = mat[i];
        for (int i = g.lane; i < n; i += 32) piv[s * n + i] = pv[i];
        if (g.lane == 0) info[s] = ok ? 0 : bad + 1;
        g.sync();
    }
}


// ---------------------------------------------------------------- adjoint
// Discrete adjoint of the recorded forward map (a lane group per cell, FP64).
// Replay: recompute the step history from the tape header (y0, h0) with each
// corrector solved to rounding level (Newton with the analytic Jacobian at
// the recorded state, the matrix in FP32 and the residual in FP64),
// overwriting the tape's states with these exact ones.
// Reverse: lam (the adjoint of the Nordsieck array) is carried back through
// each step's update, corrector (mu = (I - gamma J(y_n))^{-T} lam_Delta),
// prediction and column map, accumulating gamma (df/dtheta)^T mu for
// theta = (ln A_j, Ea_j): <df/dlnA_j, mu> = (q_j/rho)(sum_k nu_kj W_k mu_k
// - T dH_j mu_T / cpm), df/dEa_j = -df/dlnA_j / (Rc T).
struct AdjArgs {
    MechArgs m;
    const double *dLdy;     // [C, N]
    double *yrep;           // [C, N] replayed final states (nullable)
    double *gcells;         // [C, M, 2]
    long long n;
};

template <int L>
__device__ void adj_theta(GroupCell<L, double> &c, const double *mu, double scale, double *g)
{
    const int K = c.K, M = c.M;
    for (int k = c.g.lane; k < K; k += L) c.wmu[k] = c.tb.W[k] * mu[k];
    c.g.sync();
    const double T = c.last_T, muT = mu[K];
    const double a = scale / c.last_rho, b = T * muT / c.last_cpm;
    const double iRT = rcp(RC * T);
    for (int j = c.g.lane; j < M; j += L) {
        const uint32_t u = c.tb.ridx[2 * j], v = c.tb.ridx[2 * j + 1];
        const int r0 = u & 0xff, r1 = (u >> 8) & 0xff, r2 = (u >> 16) & 0xff, p0 = u >> 24;
        const int p1 = v & 0xff, p2 = (v >> 8) & 0xff;
        const double sw = (c.wmu[p0] + c.wmu[p1] + c.wmu[p2]) - (c.wmu[r0] + c.wmu[r1] + c.wmu[r2]);
        const double dH = (c.hRT[p0] + c.hRT[p1] + c.hRT[p2]) - (c.hRT[r0] + c.hRT[r1] + c.hRT[r2]);
        const double d = a * c.q[j] * (sw - b * dH);
        g[2 * j] += d;
        g[2 * j + 1] -= d * iRT;
    }
    c.g.sync();
}

template <int L, typename MT>
__device__ void adj_bind(GroupCell<L, MT> &c, unsigned char *smem, const MechArgs &m, int gid)
{
    c.g.lane = threadIdx.x % L;
    c.g.mask = group_mask<L>();
    c.tb = mech_tab_at(smem, m.off);
    c.N = m.off.N; c.K = m.off.K; c.M = m.off.M;
    c.invN = m.invN;
    c.bind(smem + m.off.bytes + gid * m.lay.bytes, m.lay);
    c.tape = nullptr;
}

template <int L, typename MT>
__global__ void __launch_bounds__(256) adjoint_replay_kernel(const AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    stage_bytes(smem, a.m.tab, a.m.off.bytes);
    __syncthreads();
    GroupCell<L, MT> c;
    adj_bind<L, MT>(c, smem, a.m, threadIdx.x / L);
    const int N = c.N, H = tape_header(N), R = tape_record(N);
    for (;;) {
        const long long cell = grab_group(a.m.queue, c.g.lane, c.g.mask, L);
        if (cell >= a.n) break;
        double *tp = a.m.tape + cell * a.m.tape_stride;
        c.P = a.m.p_mech[cell];
        c.invP = rcp(c.P);
        const int count = (int)tp[0];
        const bool bad = tp[2] != 0.0;
        double *z0 = c.V(V_Z0), *y = c.V(V_Y), *f = c.V(V_F), *d = c.V(V_DEL);
        for (int i = c.g.lane; i < N; i += L) y[i] = tp[8 + i];
        c.g.sync();
        c.rhs(V_Y, V_F);
        for (int i = c.g.lane; i < N; i += L) {
            z0[i] = y[i];
            c.vec[c.NP + i] = tp[1] * f[i];
            for (int j = 2; j <= QMAX; ++j) c.vec[j * c.NP + i] = 0.0;
        }
        c.g.sync();
        for (int r = 0; r < count && !bad; ++r) {
            double *rec = tp + H + (long long)r * R;
            const double *Pm = rec + N, *cv = rec + N + 36;
            const double gamma = rec[N + 42], il1 = rec[N + 43];
            const int q = (int)rec[N + 44], qo = (int)rec[N + 45];
            for (int i = c.g.lane; i < N; i += L) {      // Z_pre = P Z
                double zin[6], zo[6];
                for (int j = 0; j < 6; ++j) zin[j] = c.vec[j * c.NP + i];
                for (int o = 0; o < 6; ++o) {
                    double acc = 0.0;
                    for (int j = 0; j < 6; ++j) acc += Pm[o * 6 + j] * zin[j];
                    zo[o] = acc;
                }
                for (int o = 0; o < 6; ++o) c.vec[o * c.NP + i] = zo[o];
                y[i] = rec[i];
            }
            c.g.sync();
            c.predict(q);
            // Newton to rounding level with the matrix at the recorded state
            // (already within the forward Newton tolerance of the exact
            // corrector, so the iteration contracts by orders of magnitude
            // per step); f is re-evaluated every iteration
            c.eval(V_Y, V_F, gamma, true);
            const int have = c.factor();
            for (int it = 0; it < 20 && have; ++it) {
                if (it > 0) c.rhs(V_Y, V_F);
                for (int i = c.g.lane; i < N; i += L)
                    d[i] = -(y[i] - gamma * f[i] - (z0[i] - il1 * c.vec[c.NP + i]));
                c.g.sync();
                c.solve(V_DEL);
                double worst = 0.0;           // converged in every component
                for (int i = c.g.lane; i < N; i += L) {
                    y[i] += d[i];
                    worst = fmax(worst, fabs(d[i]) - (1e-13 * fabs(y[i]) + 1e-30));
                }
                worst = c.g.max(worst);
                c.g.sync();
                if (worst <= 0.0) break;
            }
            for (int i = c.g.lane; i < N; i += L) {
                rec[i] = y[i];
                const double del = y[i] - z0[i];
                for (int j = 0; j < 6; ++j) {
                    const double zj = (j <= q) ? c.vec[j * c.NP + i] : 0.0;
                    c.vec[j * c.NP + i] = (j <= qo) ? zj + cv[j] * del : 0.0;
                }
            }
            c.g.sync();
        }
        if (a.yrep)
            for (int i = c.g.lane; i < N; i += L) a.yrep[cell * N + i] = bad ? __longlong_as_double(0x7ff8000000000000LL) : z0[i];
        c.g.sync();
    }
}

template <int L>
__global__ void __launch_bounds__(256) adjoint_reverse_kernel(const AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    stage_bytes(smem, a.m.tab, a.m.off.bytes);
    __syncthreads();
    GroupCell<L, double> c;
    adj_bind<L, double>(c, smem, a.m, threadIdx.x / L);
    const int N = c.N, M = c.M, H = tape_header(N), R = tape_record(N);
    for (;;) {
        const long long cell = grab_group(a.m.queue, c.g.lane, c.g.mask, L);
        if (cell >= a.n) break;
        const double *tp = a.m.tape + cell * a.m.tape_stride;
        double *g = a.gcells + cell * 2 * M;
        for (int j = c.g.lane; j < 2 * M; j += L) g[j] = 0.0;
        c.P = a.m.p_mech[cell];
        c.invP = rcp(c.P);
        const int count = (int)tp[0];
        const bool bad = tp[2] != 0.0;
        double *lam = c.vec, *y = c.V(V_Y), *ld = c.V(V_DEL);
        for (int i = c.g.lane; i < N; i += L) {
            lam[i] = a.dLdy[cell * N + i];
            for (int j = 1; j < 6; ++j) lam[j * c.NP + i] = 0.0;
        }
        c.g.sync();
        for (int r = count - 1; r >= 0 && !bad; --r) {
            const double *rec = tp + H + (long long)r * R;
            const double *Pm = rec + N, *cv = rec + N + 36;
            const double gamma = rec[N + 42], il1 = rec[N + 43];
            const int q = (int)rec[N + 44], qo = (int)rec[N + 45];
            for (int i = c.g.lane; i < N; i += L) {
                double s = 0.0;
                for (int j = 0; j <= qo; ++j) s += cv[j] * lam[j * c.NP + i];
                ld[i] = s;
                for (int j = q + 1; j < 6; ++j) lam[j * c.NP + i] = 0.0;
                lam[i] -= s;
                y[i] = rec[i];
            }
            c.g.sync();
            c.eval(V_Y, V_F, gamma, true);       // M = I - gamma J(y_n)
            c.factor();
            lu_solve_t<L>(c.g, c.mat, N, c.perm, c.dinv, c.xs, ld);   // mu
            adj_theta<L>(c, ld, gamma, g);
            for (int i = c.g.lane; i < N; i += L) {
                lam[i] += ld[i];
                lam[c.NP + i] -= il1 * ld[i];
                double l6[6], o6[6];
                for (int j = 0; j < 6; ++j) l6[j] = lam[j * c.NP + i];
                for (int k = q - 1; k >= 0; --k)              // prediction, transposed
                    for (int j = k + 1; j <= q; ++j) l6[j] += l6[j - 1];
                for (int aa = 0; aa < 6; ++aa) {              // column map, transposed
                    double acc = 0.0;
                    for (int o = 0; o < 6; ++o) acc += Pm[o * 6 + aa] * l6[o];
                    o6[aa] = acc;
                }
                for (int j = 0; j < 6; ++j) lam[j * c.NP + i] = o6[j];
            }
            c.g.sync();
        }
        // z1 = h0 f(y0)
        for (int i = c.g.lane; i < N; i += L) y[i] = tp[8 + i];
        c.g.sync();
        c.rhs(V_Y, V_F);
        if (!bad) adj_theta<L>(c, lam + c.NP, tp[1], g);
        else
            for (int j = c.g.lane; j < 2 * M; j += L) g[j] = __longlong_as_double(0x7ff8000000000000LL);
        c.g.sync();
    }
}

// Deterministic sum over cells: fixed chunks, then the chunk sums in order.
__global__ void grad_partial_kernel(const double *gcells, long long n, int len, int chunk, double *part)
{
    const int t = threadIdx.x + blockIdx.y * blockDim.x;
    if (t >= len) return;
    const long long c0 = (long long)blockIdx.x * chunk;
    const long long c1 = c0 + chunk < n ? c0 + chunk : n;
    double s = 0.0;
    for (long long cc = c0; cc < c1; ++cc) s += gcells[cc * len + t];
    part[(long long)blockIdx.x * len + t] = s;
}

__global__ void grad_final_kernel(const double *part, int nchunks, int len, double *grad)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len) return;
    double s = 0.0;
    for (int k = 0; k < nchunks; ++k) s += part[(long long)k * len + t];
    grad[t] = s;
}

struct DevTotals {
    unsigned long long sum[6];
    int max_nst;
    int worst;
    unsigned long long nfail;
};

__global__ void totals_kernel(const int32_t *stats, long long n, DevTotals *t)
{
    unsigned long long s[6] = {0, 0, 0, 0, 0, 0}, nf = 0;
    int mx = 0, worst = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int4 a = reinterpret_cast<const int4 *>(stats)[2 * c];
        const int4 b = reinterpret_cast<const int4 *>(stats)[2 * c + 1];
        s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w; s[4] += b.x; s[5] += b.y;
        mx = max(mx, a.x);
        worst = min(worst, b.w);
        nf += (b.w != 0);
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        worst = min(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < 6; ++i) atomicAdd(&t->sum[i], s[i]);
        atomicAdd(&t->nfail, nf);
        atomicMax(&t->max_nst, mx);
        atomicMin(&t->worst, worst);
    }
}

// ============================================================ host side

// The right-hand sides' logarithm on a device array, for its accuracy test.
__global__ void log_check_kernel(const double *x, double *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = flog(x[i]);
}

// The right-hand sides' exponential on a device array, for its accuracy test.
__global__ void exp_check_kernel(const double *x, double *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fexp(x[i], g_exp_tab);
}

// Typical values (Sec. 4.1.3): per component the minimum and maximum over
// the cells, as order-preserving 64-bit keys (sign-magnitude flipped to
// two's order) so that the atomics are exact and order-independent.
__device__ __forceinline__ unsigned long long order_key(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// block (x, i): component i of cells x, x + gridDim.x, ... of y [C, n]
// (comp0 + i indexes keys: minima at [k], maxima at [KEYS_MAX + k])
constexpr int KEYS_MAX = 128;
__global__ void __launch_bounds__(256) typical_minmax_kernel(const double *y, long long C, int n, int comp0,
                                                             unsigned long long *keys)
{
    const int i = blockIdx.y;
    unsigned long long mn = ~0ull, mx = 0ull;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = order_key(y[c * n + i]);
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(keys + comp0 + i, mn);
        atomicMax(keys + KEYS_MAX + comp0 + i, mx);
    }
}

// One kernel launch of an outer step.
struct LaunchSpec {
    void *func = nullptr;
    dim3 grid, block;
    int smem = 0;
    bool thread = false;    // arguments in ta (thread kernel) or ma (mechanism kernel)
    MechArgs ma{};
    ThreadArgs ta{};
    void *arg() { return thread ? (void *)&ta : (void *)&ma; }
};

struct sunb_ctx {
    int kind = 0;
    long long C = 0, Cc = 0;         // mechanism (or Robertson/cosmology) cells, cosmology cells (mixed)
    int N = 0;
    int max_order = 5, max_steps = 100000, precision = SUNB_FP64, L = 32, schedule = SUNB_SCHED_QUEUE;
    bool autotune = false, tuned = false;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 148;
    double rtol = 1e-6;
    std::vector<double> atol;        // N (+1 for mixed)
    const double *params = nullptr;
    // mechanism
    MechTabOffsets off{};
    std::vector<unsigned char> blob;
    unsigned char *d_tab = nullptr;
    CellLayout lay{};
    int cells_per_cta = 1, ctas_per_sm = 1;
    // cosmology
    double *d_cool = nullptr;
    int nknots = 0;
    double gamma_heat = 0.0;
    int jac_dq = 0;                  // mechanism Newton matrix: 0 analytic, 1 difference quotients
    int lin_solver = 0;              // mechanism linear solves: 0 LU, 1 GMRES
    int method = 0;                  // thread-per-cell kinds: SUNB_METHOD_BDF or SUNB_METHOD_ERK
    double *d_krylov = nullptr;      // GMRES scratch, one block per resident lane group
    size_t krylov_cap = 0;           // its size in doubles
    // workspace
    int32_t *d_stats = nullptr;
    unsigned long long *d_queue = nullptr;
    unsigned long long *d_minmax = nullptr;   // typical-value keys (2 x KEYS_MAX)
    DevTotals *d_totals = nullptr;
    double *d_ybuf = nullptr;
    int32_t *d_sbuf = nullptr;
    double *d_tune = nullptr;        // autotuning sample (copy of the first cells)
    double *d_tape = nullptr;        // adjoint tapes, one per mechanism cell
    long long tape_stride = 0;
    int tape_cap = 0;
    bool replayed = false;           // tapes hold exact states of the last integration
    double *d_gcells = nullptr;      // per-cell gradients [C, M, 2]
    // CUDA graph of captured outer steps
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<cudaGraphNode_t> graph_kernels;    // kernel nodes, step-major
    std::vector<LaunchSpec> graph_specs;          // their launches, same order
    std::vector<int> graph_step;                  // the outer step of each node
    double graph_dt = 0.0;
    double *d_gpart = nullptr;       // partial sums of the gradient reduction
    long long tune_cells = 0;
    float tune_ms[3][2] = {{0}};     // per L = 8/16/32: trial ms and trial cells
    long long launches = 0;
    std::string err;
};

static std::string g_create_error = "no error";

// Message for sunb_last_error(NULL) from entry points that have no context.
void sunb_internal_set_error(const std::string &msg) { g_create_error = msg; }

static int fail(sunb_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg; else g_create_error = msg;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, SUNB_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int align16(int x) { return (x + 15) & ~15; }

static int build_mech_blob(sunb_ctx *ctx, const sunb_mechanism *m)
{
    const int K = m->n_species, M = m->n_reactions, N = K + 1;
    if (K < 1 || K > 63 || M < 1 || M > 4096)
        return fail(ctx, SUNB_ILL_INPUT, "mechanism: need 1 <= n_species <= 63 and 1 <= n_reactions <= 4096");
    if (!m->W || !m->nasa || !m->react || !m->prod || !m->lnA || !m->beta || !m->Ea)
        return fail(ctx, SUNB_ILL_INPUT, "mechanism: a table pointer is NULL");
    std::vector<std::vector<std::pair<int, int>>> inc(K);
    std::vector<uint32_t> ridx(2 * M);
    for (int j = 0; j < M; ++j) {
        int r[3], p[3], nr = 0, np = 0;
        for (int s = 0; s < 3; ++s) {
            r[s] = m->react[3 * j + s];
            p[s] = m->prod[3 * j + s];
            if (r[s] < -1 || r[s] >= K || p[s] < -1 || p[s] >= K)
                return fail(ctx, SUNB_ILL_INPUT, "mechanism: species index out of range in reaction " + std::to_string(j));
            nr += r[s] >= 0;
            np += p[s] >= 0;
        }
        if (nr == 0 || np == 0)
            return fail(ctx, SUNB_ILL_INPUT, "mechanism: reaction " + std::to_string(j) + " lacks reactants or products");
        int rs[3], ps[3];
        for (int s = 0; s < 3; ++s) { rs[s] = r[s] >= 0 ? r[s] : K; ps[s] = p[s] >= 0 ? p[s] : K; }
        // keep used slots first so that position 0 is always a species
        std::stable_partition(rs, rs + 3, [K](int v) { return v != K; });
        std::stable_partition(ps, ps + 3, [K](int v) { return v != K; });
        const int dnu = np - nr;
        ridx[2 * j] = (uint32_t)rs[0] | ((uint32_t)rs[1] << 8) | ((uint32_t)rs[2] << 16) | ((uint32_t)ps[0] << 24);
        ridx[2 * j + 1] = (uint32_t)ps[1] | ((uint32_t)ps[2] << 8) | ((uint32_t)(dnu + 8) << 16) |
                          ((uint32_t)nr << 24);
        int net[64] = {0};
        for (int s = 0; s < 3; ++s) {
            if (r[s] >= 0) net[r[s]] -= 1;
            if (p[s] >= 0) net[p[s]] += 1;
        }
        for (int k = 0; k < K; ++k)
            if (net[k] != 0) inc[k].push_back({j, net[k]});
    }
    int nnz = 0;
    for (int k = 0; k < K; ++k) nnz += (int)inc[k].size();

    MechTabOffsets o{};
    o.K = K; o.M = M; o.N = N; o.nnz = nnz;
    int off = 0;
    auto take = [&](int bytes) { const int r = off; off = align16(off + bytes); return r; };
    o.invW = take(8 * K); o.W = take(8 * K); o.cpc = take(8 * 5 * K); o.hc = take(8 * 6 * K);
    o.sc = take(8 * 6 * K); o.dcp = take(8 * 4 * K); o.rpar = take(8 * 3 * M); o.atol = take(8 * N);
    o.inc_nu = take(8 * std::max(nnz, 1)); o.ridx = take(4 * 2 * M); o.inc_ptr = take(4 * (K + 1));
    o.inc_j = take(4 * std::max(nnz, 1));
    o.inc_nuf = take(4 * std::max(nnz, 1));
    o.invWf = take(4 * K);
    o.exptab = take(8 * EXP_TABLE_SIZE);
    o.bytes = off;
    std::vector<unsigned char> blob(off, 0);
    auto D = [&](int o_) { return reinterpret_cast<double *>(blob.data() + o_); };
    auto I = [&](int o_) { return reinterpret_cast<int32_t *>(blob.data() + o_); };
    for (int k = 0; k < K; ++k) {
        const double *a = m->nasa + 7 * k;
        if (!(m->W[k] > 0.0)) return fail(ctx, SUNB_ILL_INPUT, "mechanism: molecular weights must be positive");
        D(o.invW)[k] = 1.0 / m->W[k];
        D(o.W)[k] = m->W[k];
        for (int i = 0; i < 5; ++i) D(o.cpc)[5 * k + i] = a[i];
        const double hc[6] = {a[0], a[1] / 2.0, a[2] / 3.0, a[3] / 4.0, a[4] / 5.0, a[5]};
        const double sc[6] = {a[0], a[1], a[2] / 2.0, a[3] / 3.0, a[4] / 4.0, a[6]};
        const double dc[4] = {a[1], 2.0 * a[2], 3.0 * a[3], 4.0 * a[4]};
        for (int i = 0; i < 6; ++i) { D(o.hc)[6 * k + i] = hc[i]; D(o.sc)[6 * k + i] = sc[i]; }
        for (int i = 0; i < 4; ++i) D(o.dcp)[4 * k + i] = dc[i];
    }
    for (int j = 0; j < M; ++j) {
        D(o.rpar)[3 * j] = m->lnA[j];
        D(o.rpar)[3 * j + 1] = m->beta[j];
        D(o.rpar)[3 * j + 2] = m->Ea[j] / RC;
    }
    for (int i = 0; i < N; ++i) D(o.atol)[i] = 1e-10;
    int e = 0;
    for (int k = 0; k < K; ++k) {
        I(o.inc_ptr)[k] = e;
        for (auto &pr : inc[k]) {
            I(o.inc_j)[e] = pr.first;
            D(o.inc_nu)[e] = (double)pr.second;
            reinterpret_cast<float *>(blob.data() + o.inc_nuf)[e] = (float)pr.second;
            ++e;
        }
        reinterpret_cast<float *>(blob.data() + o.invWf)[k] = (float)(1.0 / m->W[k]);
    }
    I(o.inc_ptr)[K] = e;
    std::memcpy(blob.data() + o.ridx, ridx.data(), 4 * 2 * M);
    exp_table_values(D(o.exptab));
    ctx->off = o;
    ctx->blob.swap(blob);
    return SUNB_SUCCESS;
}

// Bytes of one Newton-matrix scratch: dq [6M] in the matrix type, then
// dqdT and uq [M] and wdot, u, wT [K] in FP64 (GroupCell::set_jac_scratch).
static int jac_scratch_bytes(int M, int K, int mt) { return align16(mt * 6 * M) + 16 * M + 24 * K; }

static CellLayout make_layout(int N, int K, int M, int mt, bool dq_in_cell = true, bool with_pm = true)
{
    CellLayout l{};
    l.NP = (N + 1) & ~1;
    int off = 0;
    auto take = [&](int bytes) { const int r = off; off = align16(off + bytes); return r; };
    l.vec = take(8 * NVEC * l.NP);
    l.mat = take(mt * N * N);
    l.perm = take(4 * N);
    l.xs = take(mt * 2 * N);
    l.sp = take(8 * (4 * (K + 1) + K));
    l.rq = take(8 * M);
    l.dq = dq_in_cell ? take(jac_scratch_bytes(M, K, mt)) : -1;
    l.pm = with_pm ? take(8 * (36 + K + 1)) : -1;   // adjoint column map and scratch
    l.bytes = off;
    return l;
}

// The cell fields of a layout moved by shift bytes (cells placed after the
// cooling table of a mixed launch).
static CellLayout shifted(CellLayout l, int shift)
{
    l.vec += shift; l.mat += shift; l.perm += shift; l.xs += shift;
    l.sp += shift; l.rq += shift;
    if (l.dq >= 0) l.dq += shift;
    if (l.pm >= 0) l.pm += shift;
    return l;
}

template <int L, typename MT, bool COSMO>
static void *mech_kernel_ptr(bool krylov)
{
    return krylov ? (void *)mech_kernel<L, MT, COSMO, true> : (void *)mech_kernel<L, MT, COSMO, false>;
}

static void *pick_mech_kernel(int L, int precision, bool cosmo, bool krylov)
{
    const bool f = precision == SUNB_MIXED32;
#define PICK(LL)                                                                                   \
    if (L == LL) return f ? (cosmo ? mech_kernel_ptr<LL, float, true>(krylov) : mech_kernel_ptr<LL, float, false>(krylov)) \
                          : (cosmo ? mech_kernel_ptr<LL, double, true>(krylov) : mech_kernel_ptr<LL, double, false>(krylov));
    PICK(8) PICK(16) PICK(32)
#undef PICK
    return nullptr;
}

static int cool_bytes(const sunb_ctx *c) { return c->nknots ? align16(cooling_smem_bytes(c->nknots)) : 0; }

// Shared memory of a mechanism CTA with c cells of L lanes: the tables, the
// cooling table (mixed launches), the cells, one Newton-matrix scratch per
// warp, and the warps' scratch locks.
struct MechSmem {
    int cells_off, dq_off, dq_bytes, lock_off, bytes;
};
static MechSmem mech_smem(const sunb_ctx *ctx, int c, int L)
{
    MechSmem m;
    const int mt = ctx->precision == SUNB_MIXED32 ? 4 : 8;
    const int warps = (c * L + 31) / 32;
    m.cells_off = ctx->off.bytes + (ctx->kind == SUNB_MIXED ? cool_bytes(ctx) : 0);
    m.dq_bytes = jac_scratch_bytes(ctx->off.M, ctx->off.K, mt);
    m.dq_off = m.cells_off + c * ctx->lay.bytes;
    m.lock_off = m.dq_off + warps * m.dq_bytes;
    m.bytes = m.lock_off + align16(4 * warps);
    return m;
}

// GMRES scratch for every lane group of a mechanism launch (grid of
// num_sms x ctas_per_sm CTAs of cells_per_cta groups), grown when a
// configuration needs more; nothing without the Krylov solver.
static int ensure_krylov(sunb_ctx *ctx)
{
    if (ctx->lin_solver != 1) return SUNB_SUCCESS;
    const size_t need = (size_t)ctx->num_sms * ctx->ctas_per_sm * ctx->cells_per_cta * krylov_doubles(ctx->off.N);
    if (need <= ctx->krylov_cap) return SUNB_SUCCESS;
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->d_krylov) cudaFree(ctx->d_krylov);
    ctx->d_krylov = nullptr;
    ctx->krylov_cap = 0;
    if (cudaMalloc(&ctx->d_krylov, 8 * need) != cudaSuccess) {
        cudaGetLastError();
        ctx->d_krylov = nullptr;
        return fail(ctx, SUNB_MEM_FAIL, "GMRES scratch: device allocation failed");
    }
    ctx->krylov_cap = need;
    return SUNB_SUCCESS;
}

// Whether a mechanism launch of the current configuration may run: the
// Krylov kernel needs scratch for every lane group of its grid.
static int krylov_ready(sunb_ctx *ctx)
{
    if (ctx->lin_solver != 1) return SUNB_SUCCESS;
    const size_t need = (size_t)ctx->num_sms * ctx->ctas_per_sm * ctx->cells_per_cta * krylov_doubles(ctx->off.N);
    if (ctx->d_krylov && ctx->krylov_cap >= need) return SUNB_SUCCESS;
    return fail(ctx, SUNB_MEM_FAIL, "GMRES scratch missing for this configuration");
}

// Cells per CTA for lanes-per-cell L: the count that keeps the most cells
// resident per SM within the shared-memory budget (whole warps, <= 256 threads).
static int configure_mech(sunb_ctx *ctx, int L, int force_cpc = 0)
{
    const int mt = ctx->precision == SUNB_MIXED32 ? 4 : 8;
    ctx->lay = make_layout(ctx->off.N, ctx->off.K, ctx->off.M, mt, false, ctx->tape_cap > 0);
    const bool cosmo = ctx->kind == SUNB_MIXED;
    int dev_optin = 0, sm_bytes = 0;
    CU(cudaDeviceGetAttribute(&dev_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    CU(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    int best_c = 0, best_res = -1;
    for (int c = std::max(1, 32 / L); c * L <= 256; c += std::max(1, 32 / L)) {
        const int bytes = mech_smem(ctx, c, L).bytes;
        if (bytes > dev_optin) break;
        int blocks = sm_bytes / (bytes + 1024);
        blocks = std::min(blocks, 2048 / (c * L));
        const int res = blocks * c;
        if (res > best_res) { best_res = res; best_c = c; }
    }
    if (best_c == 0)
        return fail(ctx, SUNB_ILL_INPUT, "mechanism too large for shared memory at this precision and mapping");
    if (force_cpc > 0) {
        if (force_cpc * L > 256 || (force_cpc * L) % 32 != 0 || mech_smem(ctx, force_cpc, L).bytes > dev_optin)
            return fail(ctx, SUNB_ILL_INPUT, "cells per CTA does not fit");
        best_c = force_cpc;
    }
    ctx->L = L;
    ctx->cells_per_cta = best_c;
    const int bytes = mech_smem(ctx, best_c, L).bytes;
    void *k = pick_mech_kernel(L, ctx->precision, cosmo, ctx->lin_solver == 1);
    CU(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, best_c * L, bytes));
    ctx->ctas_per_sm = std::max(1, occ);
    return ensure_krylov(ctx);
}

static MechArgs mech_args(sunb_ctx *ctx, double *y, double t0, double tout, int32_t *status)
{
    MechArgs a{};
    a.tab = ctx->d_tab;
    a.off = ctx->off;
    a.lay = ctx->lay;
    a.cells_per_cta = ctx->cells_per_cta;
    a.schedule = ctx->schedule;
    a.invN = 1.0 / ctx->off.N;
    a.ctl.rtol = ctx->rtol;
    a.ctl.t0 = t0;
    a.ctl.tout = tout;
    a.ctl.max_steps = ctx->max_steps;
    a.ctl.max_order = ctx->max_order;
    a.queue = ctx->d_queue;
    a.tape = ctx->d_tape;
    a.tape_stride = ctx->tape_stride;
    a.tape_cap = ctx->tape_cap;
    const MechSmem ms = mech_smem(ctx, ctx->cells_per_cta, ctx->L);
    a.jac_dq = ctx->jac_dq;
    a.kry = ctx->lin_solver == 1 ? ctx->d_krylov : nullptr;
    a.kry_stride = krylov_doubles(ctx->off.N);
    a.dq_off = ms.dq_off;
    a.dq_bytes = ms.dq_bytes;
    a.lock_off = ms.lock_off;
    const bool mixed = ctx->kind == SUNB_MIXED;
    a.n_mech = ctx->C;
    a.y_mech = y ? y + (mixed ? ctx->Cc : 0) : nullptr;
    a.p_mech = ctx->params ? ctx->params + (mixed ? 2 * ctx->Cc : 0) : nullptr;
    a.stats_mech = ctx->d_stats + (mixed ? 8 * ctx->Cc : 0);
    a.status_mech = status ? status + (mixed ? ctx->Cc : 0) : nullptr;
    if (mixed) {
        a.n_cosmo = ctx->Cc;
        a.y_cosmo = y;
        a.p_cosmo = ctx->params;
        a.stats_cosmo = ctx->d_stats;
        a.status_cosmo = status;
        a.cool.knots = ctx->d_cool;
        a.cool.n = ctx->nknots;
        a.cool.gamma_heat = ctx->gamma_heat;
        a.atol_cosmo = ctx->atol[ctx->off.N];
        a.cool_smem_off = ctx->off.bytes;
        a.lay = shifted(ctx->lay, cool_bytes(ctx));   // the cells follow the cooling table
    }
    return a;
}

static int launch_mech(sunb_ctx *ctx, double *y, double t0, double tout, int32_t *status,
                       long long n_mech_override = -1)
{
    const bool cosmo = ctx->kind == SUNB_MIXED;
    const int kr = krylov_ready(ctx);
    if (kr != SUNB_SUCCESS) return kr;
    MechArgs a = mech_args(ctx, y, t0, tout, status);
    if (n_mech_override >= 0) {   // autotuning trial: mechanism cells only, from a scratch copy
        a.n_mech = n_mech_override;
        a.y_mech = y;
        a.p_mech = ctx->params + (cosmo ? 2 * ctx->Cc : 0);
        a.n_cosmo = 0;
        a.tape = nullptr;
    }
    const int bytes = mech_smem(ctx, ctx->cells_per_cta, ctx->L).bytes;
    const int threads = ctx->cells_per_cta * ctx->L;
    const int grid = ctx->num_sms * ctx->ctas_per_sm;
    CU(cudaMemsetAsync(ctx->d_queue, 0, 4 * sizeof(unsigned long long), ctx->stream));
    void *k = pick_mech_kernel(ctx->L, ctx->precision, cosmo, ctx->lin_solver == 1);
    void *args[] = {&a};
    CU(cudaLaunchKernel(k, dim3(grid), dim3(threads), args, bytes, ctx->stream));
    ctx->launches++;
    return SUNB_SUCCESS;
}

static ThreadArgs thread_args(sunb_ctx *ctx, double *y, double t0, double tout, int32_t *status)
{
    ThreadArgs a{};
    a.n = ctx->C;
    a.y = y;
    a.params = ctx->params;
    a.stats = ctx->d_stats;
    a.status = status;
    a.queue = ctx->d_queue;
    a.ctl.rtol = ctx->rtol;
    a.ctl.t0 = t0;
    a.ctl.tout = tout;
    a.ctl.max_steps = ctx->max_steps;
    a.ctl.max_order = ctx->max_order;
    for (int i = 0; i < ctx->N && i < 3; ++i) a.atol[i] = ctx->atol[i];
    a.cool.knots = ctx->d_cool;
    a.cool.n = ctx->nknots;
    a.cool.gamma_heat = ctx->gamma_heat;
    if (ctx->kind == SUNB_ROBERTSON || ctx->kind == SUNB_COSMOLOGY) {
        a.tape = ctx->d_tape;
        a.tape_stride = ctx->tape_stride;
        a.tape_cap = ctx->tape_cap;
    }
    return a;
}

template <typename MT>
static int lu_batched(int32_t n, int64_t batch, MT *A, int32_t *piv, MT *b, int32_t *info, void *stream)
{
    sunb_ctx *ctx = nullptr;
    if (n < 1 || n > 64 || batch < 0 || !A || !piv || !b || !info)
        return fail(nullptr, SUNB_ILL_INPUT, "lu: need 1 <= n <= 64 and non-NULL arrays");
    if (batch == 0) return SUNB_SUCCESS;
    const int per_warp = align16((int)sizeof(MT) * (n * n + 2 * n) + 8 * n);
    const int warps = 4;
    const int bytes = warps * per_warp;
    CU(cudaFuncSetAttribute((void *)lu_batched_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>((batch + warps - 1) / warps, 16LL * sms);
    lu_batched_kernel<MT><<<grid, 32 * warps, bytes, (cudaStream_t)stream>>>(n, batch, A, piv, b, info, per_warp);
    CU(cudaGetLastError());
    return SUNB_SUCCESS;
}


// Autotuner for the mechanism mapping (lanes per cell L and cells per CTA):
// on the first integration of a context created with lanes_per_cell = 0,
// each candidate (L = 8, 16, 32 at its resident-maximising CTA size)
// integrates a scratch copy of the first cells -- eight full waves of that
// mapping, so that the trial measures steady-state throughput rather than
// the latency of a single wave -- timed with CUDA events on the context's
// stream; the mapping with the least time per cell is kept.  The trials are
// synchronous and leave the caller's state untouched.
static long long resident_cells(sunb_ctx *ctx) { return (long long)ctx->num_sms * ctx->ctas_per_sm * ctx->cells_per_cta; }

// Two timing events, destroyed on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

static int autotune(sunb_ctx *ctx, const double *dev_y, double t0, double tout)
{
    const bool mixed = ctx->kind == SUNB_MIXED;
    const double *ysrc = dev_y + (mixed ? ctx->Cc : 0);
    EventPair ev;
    CU(cudaEventCreate(&ev.a));
    CU(cudaEventCreate(&ev.b));
    double best = 1e300;
    const int startL = ctx->L, startc = ctx->cells_per_cta;
    int bestL = startL, bestc = startc;
    const int Ls[3] = {8, 16, 32};
    // any failure inside a trial returns with the mapping it started from
    auto restore = [&](int code) -> int {
        const std::string why = ctx->err;
        configure_mech(ctx, startL, startc);
        ctx->err = why;
        return code;
    };
    auto cu = [&](cudaError_t e, const char *what) -> int {
        if (e == cudaSuccess) return SUNB_SUCCESS;
        fail(ctx, SUNB_CUDA_ERROR, std::string("autotune: ") + what + ": " + cudaGetErrorString(e));
        return restore(SUNB_CUDA_ERROR);
    };
    for (int li = 0; li < 3; ++li) {
        if (configure_mech(ctx, Ls[li]) != SUNB_SUCCESS) { ctx->tune_ms[li][0] = -1.0f; continue; }
        const long long n = std::min<long long>(ctx->tune_cells, 8 * resident_cells(ctx));
        int r;
        if ((r = cu(cudaMemcpyAsync(ctx->d_tune, ysrc, 8 * (size_t)n * ctx->N, cudaMemcpyDeviceToDevice,
                                    ctx->stream), "copy")) != SUNB_SUCCESS)
            return r;
        if ((r = cu(cudaEventRecord(ev.a, ctx->stream), "event")) != SUNB_SUCCESS) return r;
        r = launch_mech(ctx, ctx->d_tune, t0, tout, nullptr, n);
        if (r != SUNB_SUCCESS) return restore(r);
        if ((r = cu(cudaEventRecord(ev.b, ctx->stream), "event")) != SUNB_SUCCESS) return r;
        if ((r = cu(cudaEventSynchronize(ev.b), "trial")) != SUNB_SUCCESS) return r;
        float ms = 0.0f;
        if ((r = cu(cudaEventElapsedTime(&ms, ev.a, ev.b), "timing")) != SUNB_SUCCESS) return r;
        ctx->tune_ms[li][0] = ms;
        ctx->tune_ms[li][1] = (float)n;
        const double per_cell = ms / (double)n;
        if (per_cell < best) { best = per_cell; bestL = Ls[li]; bestc = ctx->cells_per_cta; }
    }
    ctx->tuned = true;
    return configure_mech(ctx, bestL, bestc);
}

// One warp per cell, up to four cells per CTA within the shared-memory limit.
static int eval_config(sunb_ctx *ctx, MechArgs &a, int &bytes)
{
    int optin = 0;
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    a.lay = make_layout(ctx->off.N, ctx->off.K, ctx->off.M, 8);
    a.cells_per_cta = 4;
    while (a.cells_per_cta > 1 && ctx->off.bytes + a.cells_per_cta * a.lay.bytes > optin) --a.cells_per_cta;
    bytes = ctx->off.bytes + a.cells_per_cta * a.lay.bytes;
    if (bytes > optin) return fail(ctx, SUNB_ILL_INPUT, "mechanism too large for the evaluation kernel");
    CU(cudaFuncSetAttribute((void *)mech_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return SUNB_SUCCESS;
}


template <int L>
static void *adj_kernel(int mode)
{
    return mode == 0 ? (void *)adjoint_replay_kernel<L, float> : (void *)adjoint_reverse_kernel<L>;
}

// Adjoint kernels: 16 lanes per cell (on B300 the replay and reverse sweep
// of mech22 cells ran 15 % faster than with 32 lanes and 40 % faster than
// with 8), FP64 layout with the Jacobian scratch in each cell, as many cells
// per CTA (whole warps, at most 256 threads) as shared memory allows.
static int adj_launch(sunb_ctx *ctx, int mode, const double *dLdy, double *yrep)
{
    constexpr int L = 16;
    AdjArgs a{};
    a.m = mech_args(ctx, nullptr, 0.0, 0.0, nullptr);
    // the replay's Newton matrix only steers an iteration whose residual is
    // formed in FP64, so it converges to the same FP64 corrector in FP32; the
    // reverse sweep's transposed solve defines the gradient: FP64
    a.m.lay = make_layout(ctx->off.N, ctx->off.K, ctx->off.M, mode == 0 ? 4 : 8);
    a.dLdy = dLdy;
    a.yrep = yrep;
    a.gcells = ctx->d_gcells;
    a.n = ctx->C;
    int optin = 0;
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    const int step = std::max(1, 32 / L);
    int cpc = 0;
    for (int c = step; c * L <= 256 && ctx->off.bytes + c * a.m.lay.bytes <= optin; c += step) cpc = c;
    if (cpc == 0) return fail(ctx, SUNB_ILL_INPUT, "mechanism too large for the adjoint kernels");
    a.m.cells_per_cta = cpc;
    const int bytes = ctx->off.bytes + cpc * a.m.lay.bytes;
    void *k = adj_kernel<L>(mode);
    CU(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int occ = 1;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, L * cpc, bytes));
    CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(unsigned long long), ctx->stream));
    void *args[] = {&a};
    CU(cudaLaunchKernel(k, dim3(ctx->num_sms * std::max(1, occ)), dim3(L * cpc), args, bytes, ctx->stream));
    ctx->launches++;
    return SUNB_SUCCESS;
}

// Thread-per-cell launch: 256 threads per CTA, as many CTAs as stay resident.
static int thread_spec(sunb_ctx *ctx, const ThreadArgs &a, bool robertson, LaunchSpec &sp,
                       bool may_spread = true)
{
    sp.thread = true;
    sp.ta = a;
    const bool erk = ctx->method == SUNB_METHOD_ERK;
    const bool rec = a.tape != nullptr;     // step-history tapes: the recording kernel
    if (rec)
        sp.func = robertson ? (void *)thread_kernel<RobertsonProblem, false, true>
                            : (void *)thread_kernel<CosmologyProblem, false, true>;
    else
        sp.func = robertson ? (erk ? (void *)thread_kernel<RobertsonProblem, true> : (void *)thread_kernel<RobertsonProblem>)
                            : (erk ? (void *)thread_kernel<CosmologyProblem, true> : (void *)thread_kernel<CosmologyProblem>);
    sp.smem = 0;
    // A batch of at most 256 cells per SM runs as one wave spread over every
    // SM, at most 8 warps of about 2 cells each per SM: 1024 Robertson cells
    // took 22.1 ms on 4 SMs from the queue, 10.0 ms as 1 warp of 7 cells per
    // SM, 8.7 ms as 7 warps of 1 cell and 7.8 ms as 4 warps of 2 (B300).
    constexpr int SPREAD_LANES = 2, SPREAD_WARPS = 8;
    const long long per_sm = (a.n + ctx->num_sms - 1) / ctx->num_sms;
    if (may_spread && per_sm <= (long long)SPREAD_WARPS * 32) {
        const int W = (int)std::min<long long>(SPREAD_WARPS, (per_sm + SPREAD_LANES - 1) / SPREAD_LANES);
        sp.ta.spread_lanes = (int)((per_sm + W - 1) / W);
        sp.grid = dim3((unsigned)ctx->num_sms);
        sp.block = dim3(32 * std::max(1, W));
        return SUNB_SUCCESS;
    }
    sp.ta.spread_lanes = 0;
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sp.func, 256, 0));
    const long long want = (a.n + 255) / 256;
    sp.grid = dim3((unsigned)std::max(1LL, std::min<long long>(want, (long long)ctx->num_sms * std::max(1, occ))));
    sp.block = dim3(256);
    return SUNB_SUCCESS;
}

// The kernel launches of one outer step, which follow a reset of the cell
// counters: one kernel, or for a mixed batch the mechanism kernel (with
// cosmology cells in its tail) and then the cosmology thread kernel, which
// takes the cosmology cells that are left from the same counter.
static int step_config(sunb_ctx *ctx, double *y, double t0, double tout, int32_t *status, LaunchSpec sp[2],
                       int &n)
{
    n = 0;
    if (ctx->kind == SUNB_ROBERTSON || ctx->kind == SUNB_COSMOLOGY) {
        n = 1;
        return thread_spec(ctx, thread_args(ctx, y, t0, tout, status), ctx->kind == SUNB_ROBERTSON, sp[0]);
    }
    const bool cosmo = ctx->kind == SUNB_MIXED;
    LaunchSpec &m = sp[0];
    m.thread = false;
    const int kr = krylov_ready(ctx);
    if (kr != SUNB_SUCCESS) return kr;
    m.ma = mech_args(ctx, y, t0, tout, status);
    m.func = pick_mech_kernel(ctx->L, ctx->precision, cosmo, ctx->lin_solver == 1);
    m.smem = mech_smem(ctx, ctx->cells_per_cta, ctx->L).bytes;
    m.grid = dim3(ctx->num_sms * ctx->ctas_per_sm);
    m.block = dim3(ctx->cells_per_cta * ctx->L);
    n = 1;
    if (cosmo) {
        ThreadArgs ta = thread_args(ctx, y, t0, tout, status);
        ta.n = ctx->Cc;
        ta.queue = ctx->d_queue + 1;
        ta.atol[0] = ctx->atol[ctx->off.N];
        // the queue, never the spread: the mechanism kernel's tail has
        // taken cells from the same counter
        const int rc = thread_spec(ctx, ta, false, sp[1], false);
        if (rc != SUNB_SUCCESS) return rc;
        n = 2;
    }
    return SUNB_SUCCESS;
}

static int launch_step(sunb_ctx *ctx, double *y, double t0, double tout, int32_t *status)
{
    LaunchSpec sp[2];
    int n = 0;
    const int rc = step_config(ctx, y, t0, tout, status, sp, n);
    if (rc != SUNB_SUCCESS) return rc;
    CU(cudaMemsetAsync(ctx->d_queue, 0, 4 * sizeof(unsigned long long), ctx->stream));
    for (int i = 0; i < n; ++i) {
        void *args[] = {sp[i].arg()};
        CU(cudaLaunchKernel(sp[i].func, sp[i].grid, sp[i].block, args, sp[i].smem, ctx->stream));
        ctx->launches++;
    }
    return SUNB_SUCCESS;
}

extern "C" {

const char *sunb_version(void) { return "sunb 0.1 (sm_103a)"; }

const char *sunb_last_error(const sunb_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int sunb_create(const sunb_problem *prob, void *stream, sunb_ctx **out)
{
    if (!out) return fail(nullptr, SUNB_ILL_INPUT, "out is NULL");
    *out = nullptr;
    if (!prob) return fail(nullptr, SUNB_ILL_INPUT, "problem is NULL");
    sunb_ctx *ctx = new (std::nothrow) sunb_ctx;
    if (!ctx) return fail(nullptr, SUNB_MEM_FAIL, "host allocation failed");
    auto bail = [&](int code) { g_create_error = ctx->err; sunb_destroy(ctx); return code; };
    ctx->kind = prob->kind;
    ctx->C = prob->n_cells;
    ctx->Cc = prob->kind == SUNB_MIXED ? prob->n_cells_cosmo : 0;
    ctx->max_order = prob->max_order ? prob->max_order : 5;
    ctx->max_steps = prob->max_steps ? prob->max_steps : 100000;
    ctx->precision = prob->precision;
    ctx->schedule = prob->schedule;
    ctx->stream = (cudaStream_t)stream;
    if (prob->kind < SUNB_ROBERTSON || prob->kind > SUNB_MIXED) { fail(ctx, SUNB_ILL_INPUT, "unknown kind"); return bail(SUNB_ILL_INPUT); }
    if (ctx->C < 0 || ctx->Cc < 0 || (ctx->C == 0 && ctx->Cc == 0)) { fail(ctx, SUNB_ILL_INPUT, "need at least one cell"); return bail(SUNB_ILL_INPUT); }
    if (ctx->max_order < 1 || ctx->max_order > 5) { fail(ctx, SUNB_ILL_INPUT, "max_order must be 1..5"); return bail(SUNB_ILL_INPUT); }
    if (ctx->max_steps < 1) { fail(ctx, SUNB_ILL_INPUT, "max_steps must be positive"); return bail(SUNB_ILL_INPUT); }
    if (prob->precision != SUNB_FP64 && prob->precision != SUNB_MIXED32) { fail(ctx, SUNB_ILL_INPUT, "unknown precision"); return bail(SUNB_ILL_INPUT); }
    if (prob->schedule != SUNB_SCHED_QUEUE && prob->schedule != SUNB_SCHED_STATIC) { fail(ctx, SUNB_ILL_INPUT, "unknown schedule"); return bail(SUNB_ILL_INPUT); }
    if (prob->record_adjoint < 0 || prob->record_adjoint > (1 << 20)) { fail(ctx, SUNB_ILL_INPUT, "record_adjoint must be 0..2^20 steps"); return bail(SUNB_ILL_INPUT); }
    if (prob->record_adjoint && prob->kind == SUNB_MIXED) { fail(ctx, SUNB_ILL_INPUT, "tapes are recorded for single-kind contexts"); return bail(SUNB_ILL_INPUT); }
    const int lpc = prob->lanes_per_cell;
    if (lpc != 0 && lpc != 8 && lpc != 16 && lpc != 32) { fail(ctx, SUNB_ILL_INPUT, "lanes_per_cell must be 0, 8, 16 or 32"); return bail(SUNB_ILL_INPUT); }
    int rc;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) { fail(ctx, SUNB_CUDA_ERROR, "no CUDA device"); return bail(SUNB_CUDA_ERROR); }
    if (fill_math_tables() != cudaSuccess) { fail(ctx, SUNB_CUDA_ERROR, "math table copy failed"); return bail(SUNB_CUDA_ERROR); }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);

    if (ctx->kind == SUNB_ROBERTSON) ctx->N = 3;
    if (ctx->kind == SUNB_COSMOLOGY) ctx->N = 1;
    if (ctx->kind == SUNB_MECHANISM || ctx->kind == SUNB_MIXED) {
        if (!prob->mech) { fail(ctx, SUNB_ILL_INPUT, "mechanism is NULL"); return bail(SUNB_ILL_INPUT); }
        if ((rc = build_mech_blob(ctx, prob->mech)) != SUNB_SUCCESS) return bail(rc);
        ctx->N = ctx->off.N;
    }
    if (ctx->kind == SUNB_COSMOLOGY || ctx->kind == SUNB_MIXED) {
        const sunb_cooling_table *t = prob->table;
        if (!t || !t->lnT || !t->lnLam || t->n_knots < 2 || t->n_knots > 256) {
            fail(ctx, SUNB_ILL_INPUT, "cooling table missing or with n_knots outside 2..256");
            return bail(SUNB_ILL_INPUT);
        }
        std::vector<double> k(3 * t->n_knots + EXP_TABLE_SIZE, 0.0);
        exp_table_values(k.data() + 3 * t->n_knots);
        for (int i = 0; i < t->n_knots; ++i) {
            k[i] = t->lnT[i];
            k[t->n_knots + i] = t->lnLam[i];
            if (i > 0 && !(t->lnT[i] > t->lnT[i - 1])) { fail(ctx, SUNB_ILL_INPUT, "cooling knots must increase"); return bail(SUNB_ILL_INPUT); }
        }
        for (int i = 0; i + 1 < t->n_knots; ++i)
            k[2 * t->n_knots + i] = (t->lnLam[i + 1] - t->lnLam[i]) / (t->lnT[i + 1] - t->lnT[i]);
        ctx->nknots = t->n_knots;
        ctx->gamma_heat = t->gamma_heat;
        if (cudaMalloc(&ctx->d_cool, 8 * k.size()) != cudaSuccess) { fail(ctx, SUNB_MEM_FAIL, "cudaMalloc cooling table"); return bail(SUNB_MEM_FAIL); }
        if (cudaMemcpy(ctx->d_cool, k.data(), 8 * k.size(), cudaMemcpyHostToDevice) != cudaSuccess) { fail(ctx, SUNB_CUDA_ERROR, "copy cooling table"); return bail(SUNB_CUDA_ERROR); }
    }
    ctx->atol.assign(ctx->N + (ctx->kind == SUNB_MIXED ? 1 : 0), 1e-10);
    if (prob->record_adjoint && (ctx->kind == SUNB_ROBERTSON || ctx->kind == SUNB_COSMOLOGY)) {
        // thread-per-cell kinds record the step history only (no adjoint)
        ctx->tape_cap = prob->record_adjoint;
        ctx->tape_stride = tape_header(ctx->N) + (long long)ctx->tape_cap * tape_record(ctx->N);
        if (cudaMalloc(&ctx->d_tape, 8 * (size_t)ctx->tape_stride * ctx->C) != cudaSuccess) {
            fail(ctx, SUNB_MEM_FAIL, "cudaMalloc tapes");
            return bail(SUNB_MEM_FAIL);
        }
        cudaMemset(ctx->d_tape, 0, 8 * (size_t)ctx->tape_stride * ctx->C);
    }
    const long long ncell = ctx->C + ctx->Cc;
    if (cudaMalloc(&ctx->d_stats, 32 * (size_t)ncell) != cudaSuccess ||
        cudaMalloc(&ctx->d_queue, 64) != cudaSuccess ||
        cudaMalloc(&ctx->d_minmax, 16 * KEYS_MAX) != cudaSuccess ||
        cudaMalloc(&ctx->d_totals, sizeof(DevTotals)) != cudaSuccess) {
        fail(ctx, SUNB_MEM_FAIL, "cudaMalloc workspace");
        return bail(SUNB_MEM_FAIL);
    }
    cudaMemset(ctx->d_stats, 0, 32 * (size_t)ncell);
    if (ctx->kind == SUNB_MECHANISM || ctx->kind == SUNB_MIXED) {
        if (cudaMalloc(&ctx->d_tab, ctx->off.bytes) != cudaSuccess) { fail(ctx, SUNB_MEM_FAIL, "cudaMalloc tables"); return bail(SUNB_MEM_FAIL); }
        if (cudaMemcpy(ctx->d_tab, ctx->blob.data(), ctx->off.bytes, cudaMemcpyHostToDevice) != cudaSuccess) { fail(ctx, SUNB_CUDA_ERROR, "copy tables"); return bail(SUNB_CUDA_ERROR); }
        int L = lpc ? lpc : (ctx->off.N > 32 ? 32 : 16);
        ctx->autotune = lpc == 0;
        ctx->tape_cap = prob->record_adjoint > 0 ? prob->record_adjoint : 0;   // cells keep the adjoint map
        if ((rc = configure_mech(ctx, L)) != SUNB_SUCCESS) return bail(rc);
        if (prob->record_adjoint) {
            ctx->tape_stride = tape_header(ctx->N) + (long long)ctx->tape_cap * tape_record(ctx->N);
            if (cudaMalloc(&ctx->d_tape, 8 * (size_t)ctx->tape_stride * ctx->C) != cudaSuccess ||
                cudaMalloc(&ctx->d_gcells, 8 * 2 * (size_t)ctx->off.M * ctx->C) != cudaSuccess ||
                cudaMalloc(&ctx->d_gpart, 8 * 2 * (size_t)ctx->off.M * 1024) != cudaSuccess) {
                fail(ctx, SUNB_MEM_FAIL, "cudaMalloc adjoint tapes");
                return bail(SUNB_MEM_FAIL);
            }
            cudaMemset(ctx->d_tape, 0, 8 * (size_t)ctx->tape_stride * ctx->C);
        }
        if (ctx->autotune) {
            // eight waves of the densest mapping
            long long most = 0;
            for (int Lc : {8, 16, 32})
                if (configure_mech(ctx, Lc) == SUNB_SUCCESS) most = std::max(most, resident_cells(ctx));
            if ((rc = configure_mech(ctx, L)) != SUNB_SUCCESS) return bail(rc);
            ctx->tune_cells = std::min<long long>(ctx->C, 8 * most);
            if (ctx->tune_cells >= 1 &&
                cudaMalloc(&ctx->d_tune, 8 * (size_t)ctx->tune_cells * ctx->N) != cudaSuccess) {
                fail(ctx, SUNB_MEM_FAIL, "cudaMalloc autotuning scratch");
                return bail(SUNB_MEM_FAIL);
            }
        }
    }
    *out = ctx;
    return SUNB_SUCCESS;
}

int sunb_destroy(sunb_ctx *ctx)
{
    if (!ctx) return SUNB_SUCCESS;
    cudaFree(ctx->d_tab);
    cudaFree(ctx->d_cool);
    cudaFree(ctx->d_stats);
    cudaFree(ctx->d_queue);
    cudaFree(ctx->d_minmax);
    if (ctx->d_krylov) cudaFree(ctx->d_krylov);
    cudaFree(ctx->d_totals);
    cudaFree(ctx->d_ybuf);
    cudaFree(ctx->d_sbuf);
    cudaFree(ctx->d_tune);
    cudaFree(ctx->d_tape);
    cudaFree(ctx->d_gcells);
    cudaFree(ctx->d_gpart);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    delete ctx;
    return SUNB_SUCCESS;
}

int sunb_set_tolerances(sunb_ctx *ctx, double rtol, double atol_scalar, const double *host_atol)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(ctx, SUNB_ILL_INPUT, "rtol must lie in (0, 1)");
    for (size_t i = 0; i < ctx->atol.size(); ++i) {
        const double a = host_atol ? host_atol[i] : atol_scalar;
        if (!(a > 0.0) || !std::isfinite(a)) return fail(ctx, SUNB_ILL_INPUT, "atol must be positive and finite");
        ctx->atol[i] = a;
    }
    ctx->rtol = rtol;
    if (ctx->d_tab) {
        double *at = reinterpret_cast<double *>(ctx->blob.data() + ctx->off.atol);
        for (int i = 0; i < ctx->off.N; ++i) at[i] = ctx->atol[i];
        CU(cudaMemcpyAsync(ctx->d_tab + ctx->off.atol, at, 8 * ctx->off.N, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return SUNB_SUCCESS;
}

int sunb_set_jacobian(sunb_ctx *ctx, int mode)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (mode != 0 && mode != 1) return fail(ctx, SUNB_ILL_INPUT, "jacobian mode must be 0 or 1");
    if (mode == 1 && ctx->kind != SUNB_MECHANISM && ctx->kind != SUNB_MIXED)
        return fail(ctx, SUNB_ILL_INPUT, "difference-quotient Jacobians are for mechanism cells");
    if (mode == 1 && ctx->d_tape)
        return fail(ctx, SUNB_ILL_INPUT, "the adjoint needs the analytic Jacobian");
    ctx->jac_dq = mode;
    return SUNB_SUCCESS;
}

int sunb_set_linear_solver(sunb_ctx *ctx, int solver)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (solver != SUNB_LS_DIRECT && solver != SUNB_LS_GMRES)
        return fail(ctx, SUNB_ILL_INPUT, "linear solver must be SUNB_LS_DIRECT or SUNB_LS_GMRES");
    if (solver == SUNB_LS_GMRES && ctx->kind != SUNB_MECHANISM && ctx->kind != SUNB_MIXED)
        return fail(ctx, SUNB_ILL_INPUT, "GMRES solves are for mechanism cells");
    if (solver == SUNB_LS_GMRES && ctx->d_tape)
        return fail(ctx, SUNB_ILL_INPUT, "the adjoint needs the direct solver");
    if (ctx->kind != SUNB_MECHANISM && ctx->kind != SUNB_MIXED) return SUNB_SUCCESS;   // LU, as always
    const int before = ctx->lin_solver;
    ctx->lin_solver = solver;
    // the other kernel variant: its shared-memory attribute and occupancy
    // (the same mapping), then the scratch for its resident groups; on
    // failure the previous solver stays selected
    const int rc = configure_mech(ctx, ctx->L, ctx->cells_per_cta);
    if (rc != SUNB_SUCCESS) {
        const std::string why = ctx->err;
        ctx->lin_solver = before;
        configure_mech(ctx, ctx->L, ctx->cells_per_cta);
        ctx->err = why;
    }
    return rc;
}

int sunb_set_method(sunb_ctx *ctx, int method)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (method != SUNB_METHOD_BDF && method != SUNB_METHOD_ERK)
        return fail(ctx, SUNB_ILL_INPUT, "method must be SUNB_METHOD_BDF or SUNB_METHOD_ERK");
    if (method == SUNB_METHOD_ERK && ctx->kind != SUNB_ROBERTSON && ctx->kind != SUNB_COSMOLOGY)
        return fail(ctx, SUNB_ILL_INPUT, "the explicit method is built for thread-per-cell kinds only");
    if (method == SUNB_METHOD_ERK && ctx->d_tape)
        return fail(ctx, SUNB_ILL_INPUT, "tapes record the BDF's step history");
    ctx->method = method;
    return SUNB_SUCCESS;
}

int sunb_set_typical_tolerances(sunb_ctx *ctx, const double *dev_y, double rtol, double eta,
                                double *host_atol_out)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_y) return fail(ctx, SUNB_ILL_INPUT, "y is NULL");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ctx, SUNB_ILL_INPUT, "eta must be positive and finite");
    const int nc = (int)ctx->atol.size();
    if (nc > KEYS_MAX) return fail(ctx, SUNB_ILL_INPUT, "too many components for typical values");
    CU(cudaMemsetAsync(ctx->d_minmax, 0xff, 8 * KEYS_MAX, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_minmax + KEYS_MAX, 0, 8 * KEYS_MAX, ctx->stream));
    auto reduce = [&](const double *y, long long C, int n, int comp0) -> int {
        if (C <= 0) return SUNB_SUCCESS;
        const int gx = (int)std::min<long long>((C + 255) / 256, 4LL * ctx->num_sms);
        typical_minmax_kernel<<<dim3(gx, n), 256, 0, ctx->stream>>>(y, C, n, comp0, ctx->d_minmax);
        CU(cudaGetLastError());
        ctx->launches++;
        return SUNB_SUCCESS;
    };
    int rc;
    if (ctx->kind == SUNB_MIXED) {   // cosmology cells first in y, then the mechanism cells
        if ((rc = reduce(dev_y + ctx->Cc, ctx->C, ctx->N, 0)) != SUNB_SUCCESS) return rc;
        if ((rc = reduce(dev_y, ctx->Cc, 1, ctx->N)) != SUNB_SUCCESS) return rc;
    } else {
        if ((rc = reduce(dev_y, ctx->C, ctx->N, 0)) != SUNB_SUCCESS) return rc;
    }
    unsigned long long keys[2 * KEYS_MAX];
    CU(cudaMemcpyAsync(keys, ctx->d_minmax, sizeof(keys), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const long long cells[2] = {ctx->C, ctx->Cc};
    std::vector<double> atol(nc);
    for (int i = 0; i < nc; ++i) {
        const long long C = (ctx->kind == SUNB_MIXED && i == ctx->N) ? cells[1] : cells[0];
        auto value = [](unsigned long long k) {
            const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
            double v;
            std::memcpy(&v, &b, 8);
            return v;
        };
        const double mn = value(keys[i]), mx = value(keys[KEYS_MAX + i]);
        double yt = 0.5 * (mn + mx);
        if (C < 1 || std::isnan(mn) || std::isnan(mx) || !(yt > 0.0) || !(yt <= 1.7976931348623157e308))
            yt = 1.0;                          // the paper's default typical value
        atol[i] = eta * yt;
    }
    if (host_atol_out) std::memcpy(host_atol_out, atol.data(), 8 * nc);
    return sunb_set_tolerances(ctx, rtol, 0.0, atol.data());
}

// Bytes of the per-cell parameter array of a context (sunb_set_params).
static size_t params_bytes(const sunb_ctx *ctx)
{
    switch (ctx->kind) {
    case SUNB_ROBERTSON: return 8 * 3 * (size_t)ctx->C;
    case SUNB_MECHANISM: return 8 * (size_t)ctx->C;
    case SUNB_COSMOLOGY: return 8 * 2 * (size_t)ctx->C;
    default: return 8 * (2 * (size_t)ctx->Cc + (size_t)ctx->C);
    }
}

int sunb_set_params(sunb_ctx *ctx, const double *dev_params, size_t bytes)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_params) return fail(ctx, SUNB_ILL_INPUT, "params is NULL");
    const size_t want = params_bytes(ctx);
    if (bytes != want)
        return fail(ctx, SUNB_ILL_INPUT, "params: " + std::to_string(bytes) + " bytes given, the context's cells need " +
                                             std::to_string(want));
    ctx->params = dev_params;
    return SUNB_SUCCESS;
}

int sunb_integrate(sunb_ctx *ctx, double *dev_y, double t0, double tout, int32_t *dev_status)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_y) return fail(ctx, SUNB_ILL_INPUT, "y is NULL");
    if (!ctx->params) return fail(ctx, SUNB_ILL_INPUT, "parameters not set (sunb_set_params)");
    if (!std::isfinite(t0) || !std::isfinite(tout) || tout < t0)
        return fail(ctx, SUNB_ILL_INPUT, "need finite t0 <= tout");
    if (ctx->kind == SUNB_ROBERTSON || ctx->kind == SUNB_COSMOLOGY)
        return launch_step(ctx, dev_y, t0, tout, dev_status);
    ctx->replayed = false;
    if (ctx->autotune && !ctx->tuned && ctx->tune_cells > 0 && tout > t0) {
        const int rc = autotune(ctx, dev_y, t0, tout);
        if (rc != SUNB_SUCCESS) return rc;
    }
    return launch_step(ctx, dev_y, t0, tout, dev_status);
}

int sunb_stats(sunb_ctx *ctx, sunb_stats_t *host_totals, int32_t *dev_cell_stats)
{
    if (!ctx) return SUNB_ILL_INPUT;
    const long long n = ctx->C + ctx->Cc;
    DevTotals init{};
    init.max_nst = 0;
    init.worst = 0;
    CU(cudaMemcpyAsync(ctx->d_totals, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    const int grid = (int)std::min<long long>((n + 255) / 256, 4LL * ctx->num_sms);
    totals_kernel<<<std::max(1, grid), 256, 0, ctx->stream>>>(ctx->d_stats, n, ctx->d_totals);
    CU(cudaGetLastError());
    ctx->launches++;
    DevTotals t{};
    CU(cudaMemcpyAsync(&t, ctx->d_totals, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
    if (dev_cell_stats)
        CU(cudaMemcpyAsync(dev_cell_stats, ctx->d_stats, 32 * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (host_totals) {
        host_totals->nst = (int64_t)t.sum[0];
        host_totals->nfe = (int64_t)t.sum[1];
        host_totals->nje = (int64_t)t.sum[2];
        host_totals->nni = (int64_t)t.sum[3];
        host_totals->ncf = (int64_t)t.sum[4];
        host_totals->nef = (int64_t)t.sum[5];
        host_totals->max_nst = t.max_nst;
        host_totals->worst_status = t.worst;
        host_totals->n_failed = (int64_t)t.nfail;
    }
    return t.worst;
}

int sunb_integrate_host(sunb_ctx *ctx, double *host_y, double t0, double tout, int32_t *host_status)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!host_y) return fail(ctx, SUNB_ILL_INPUT, "y is NULL");
    const size_t ny = (size_t)ctx->C * ctx->N + (size_t)ctx->Cc;
    const size_t nc = (size_t)(ctx->C + ctx->Cc);
    if (!ctx->d_ybuf || !ctx->d_sbuf) {      // both staging buffers, or neither
        if (cudaMalloc(&ctx->d_ybuf, 8 * ny) != cudaSuccess || cudaMalloc(&ctx->d_sbuf, 4 * nc) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ctx->d_ybuf);
            cudaFree(ctx->d_sbuf);
            ctx->d_ybuf = nullptr;
            ctx->d_sbuf = nullptr;
            return fail(ctx, SUNB_MEM_FAIL, "cudaMalloc staging buffer");
        }
    }
    CU(cudaMemcpyAsync(ctx->d_ybuf, host_y, 8 * ny, cudaMemcpyHostToDevice, ctx->stream));
    int rc = sunb_integrate(ctx, ctx->d_ybuf, t0, tout, host_status ? ctx->d_sbuf : nullptr);
    if (rc != SUNB_SUCCESS) return rc;
    CU(cudaMemcpyAsync(host_y, ctx->d_ybuf, 8 * ny, cudaMemcpyDeviceToHost, ctx->stream));
    if (host_status)
        CU(cudaMemcpyAsync(host_status, ctx->d_sbuf, 4 * nc, cudaMemcpyDeviceToHost, ctx->stream));
    return sunb_stats(ctx, nullptr, nullptr);
}

int sunb_rhs(sunb_ctx *ctx, const double *dev_y, double *dev_f, int64_t n_cells)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_y || !dev_f || n_cells < 0) return fail(ctx, SUNB_ILL_INPUT, "bad rhs arguments");
    if (!ctx->params) return fail(ctx, SUNB_ILL_INPUT, "parameters not set (sunb_set_params)");
    if (ctx->kind == SUNB_MIXED) return fail(ctx, SUNB_ILL_INPUT, "rhs is per kind; use a single-kind context");
    if (n_cells == 0) return SUNB_SUCCESS;
    if (ctx->kind == SUNB_MECHANISM) {
        MechArgs a = mech_args(ctx, nullptr, 0.0, 0.0, nullptr);
        int bytes = 0;
        const int rc = eval_config(ctx, a, bytes);
        if (rc != SUNB_SUCCESS) return rc;
        const int grid = (int)std::min<long long>((n_cells + a.cells_per_cta - 1) / a.cells_per_cta,
                                                  8LL * ctx->num_sms);
        mech_eval_kernel<<<grid, 32 * a.cells_per_cta, bytes, ctx->stream>>>(a, dev_y, dev_f, n_cells, 0);
    } else {
        ThreadArgs a = thread_args(ctx, nullptr, 0.0, 0.0, nullptr);
        const int grid = (int)std::min<long long>((n_cells + 127) / 128, 8LL * ctx->num_sms);
        if (ctx->kind == SUNB_ROBERTSON) thread_eval_kernel<RobertsonProblem><<<grid, 128, 0, ctx->stream>>>(a, dev_y, dev_f, n_cells, 0);
        else thread_eval_kernel<CosmologyProblem><<<grid, 128, 0, ctx->stream>>>(a, dev_y, dev_f, n_cells, 0);
    }
    CU(cudaGetLastError());
    ctx->launches++;
    return SUNB_SUCCESS;
}

int sunb_jac(sunb_ctx *ctx, const double *dev_y, double *dev_J, int64_t n_cells)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_y || !dev_J || n_cells < 0) return fail(ctx, SUNB_ILL_INPUT, "bad jac arguments");
    if (!ctx->params) return fail(ctx, SUNB_ILL_INPUT, "parameters not set (sunb_set_params)");
    if (ctx->kind == SUNB_MIXED) return fail(ctx, SUNB_ILL_INPUT, "jac is per kind; use a single-kind context");
    if (n_cells == 0) return SUNB_SUCCESS;
    if (ctx->kind == SUNB_MECHANISM) {
        MechArgs a = mech_args(ctx, nullptr, 0.0, 0.0, nullptr);
        int bytes = 0;
        const int rc = eval_config(ctx, a, bytes);
        if (rc != SUNB_SUCCESS) return rc;
        const int grid = (int)std::min<long long>((n_cells + a.cells_per_cta - 1) / a.cells_per_cta,
                                                  8LL * ctx->num_sms);
        mech_eval_kernel<<<grid, 32 * a.cells_per_cta, bytes, ctx->stream>>>(a, dev_y, dev_J, n_cells, 1);
    } else {
        ThreadArgs a = thread_args(ctx, nullptr, 0.0, 0.0, nullptr);
        const int grid = (int)std::min<long long>((n_cells + 127) / 128, 8LL * ctx->num_sms);
        if (ctx->kind == SUNB_ROBERTSON) thread_eval_kernel<RobertsonProblem><<<grid, 128, 0, ctx->stream>>>(a, dev_y, dev_J, n_cells, 1);
        else thread_eval_kernel<CosmologyProblem><<<grid, 128, 0, ctx->stream>>>(a, dev_y, dev_J, n_cells, 1);
    }
    CU(cudaGetLastError());
    ctx->launches++;
    return SUNB_SUCCESS;
}

int sunb_lu_solve_batched(int32_t n, int64_t batch, double *dev_A, int32_t *dev_piv, double *dev_b,
                          int32_t *dev_info, void *stream)
{
    return lu_batched<double>(n, batch, dev_A, dev_piv, dev_b, dev_info, stream);
}

int sunb_lu_solve_batched_f32(int32_t n, int64_t batch, float *dev_A, int32_t *dev_piv, float *dev_b,
                              int32_t *dev_info, void *stream)
{
    return lu_batched<float>(n, batch, dev_A, dev_piv, dev_b, dev_info, stream);
}


int sunb_exp_check(const double *dev_x, double *dev_y, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!dev_x || !dev_y))) {
        g_create_error = "exp_check: need n >= 0 and device arrays";
        return SUNB_ILL_INPUT;
    }
    if (n == 0) return SUNB_SUCCESS;
    if (fill_math_tables() != cudaSuccess) {
        g_create_error = "exp_check: table copy failed";
        return SUNB_CUDA_ERROR;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (int)std::min<long long>((n + 255) / 256, 148 * 8);
    exp_check_kernel<<<grid, 256, 0, st>>>(dev_x, dev_y, (long long)n);
    if (cudaGetLastError() != cudaSuccess) {
        g_create_error = "exp_check: launch failed";
        return SUNB_CUDA_ERROR;
    }
    // the host table must outlive the asynchronous copy
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        g_create_error = "exp_check: kernel failed";
        return SUNB_CUDA_ERROR;
    }
    return SUNB_SUCCESS;
}

int sunb_log_check(const double *dev_x, double *dev_y, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!dev_x || !dev_y))) {
        g_create_error = "log_check: need n >= 0 and device arrays";
        return SUNB_ILL_INPUT;
    }
    if (n == 0) return SUNB_SUCCESS;
    if (fill_math_tables() != cudaSuccess) {
        g_create_error = "log_check: table copy failed";
        return SUNB_CUDA_ERROR;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (int)std::min<long long>((n + 255) / 256, 148 * 8);
    log_check_kernel<<<grid, 256, 0, st>>>(dev_x, dev_y, (long long)n);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        g_create_error = "log_check: kernel failed";
        return SUNB_CUDA_ERROR;
    }
    return SUNB_SUCCESS;
}

int sunb_adjoint_replay(sunb_ctx *ctx, double *dev_y_final)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!ctx->d_tape) return fail(ctx, SUNB_NO_RECORD, "context created without record_adjoint");
    if (ctx->kind != SUNB_MECHANISM) return fail(ctx, SUNB_ILL_INPUT, "the adjoint is for mechanism contexts");
    if (!ctx->params) return fail(ctx, SUNB_ILL_INPUT, "parameters not set (sunb_set_params)");
    const int rc = adj_launch(ctx, 0, nullptr, dev_y_final);
    if (rc == SUNB_SUCCESS) ctx->replayed = true;
    return rc;
}

int sunb_adjoint(sunb_ctx *ctx, const double *dev_dLdy, double *dev_grad, double *dev_grad_cells)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!ctx->d_tape) return fail(ctx, SUNB_NO_RECORD, "context created without record_adjoint");
    if (ctx->kind != SUNB_MECHANISM) return fail(ctx, SUNB_ILL_INPUT, "the adjoint is for mechanism contexts");
    if (!dev_dLdy || !dev_grad) return fail(ctx, SUNB_ILL_INPUT, "dLdy and grad must not be NULL");
    if (!ctx->replayed) {
        const int rc = sunb_adjoint_replay(ctx, nullptr);
        if (rc != SUNB_SUCCESS) return rc;
    }
    int rc = adj_launch(ctx, 1, dev_dLdy, nullptr);
    if (rc != SUNB_SUCCESS) return rc;
    const int len = 2 * ctx->off.M;
    const long long chunk = std::max<long long>(1, (ctx->C + 1023) / 1024);
    const int nchunks = (int)((ctx->C + chunk - 1) / chunk);
    dim3 grid(nchunks, (len + 255) / 256);
    grad_partial_kernel<<<grid, 256, 0, ctx->stream>>>(ctx->d_gcells, ctx->C, len, (int)chunk, ctx->d_gpart);
    grad_final_kernel<<<(len + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_gpart, nchunks, len, dev_grad);
    CU(cudaGetLastError());
    ctx->launches += 2;
    if (dev_grad_cells)
        CU(cudaMemcpyAsync(dev_grad_cells, ctx->d_gcells, 8 * (size_t)len * ctx->C, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    return SUNB_SUCCESS;
}

int sunb_set_arrhenius(sunb_ctx *ctx, const double *host_lnA, const double *host_Ea)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!ctx->d_tab) return fail(ctx, SUNB_ILL_INPUT, "not a mechanism context");
    if (!host_lnA || !host_Ea) return fail(ctx, SUNB_ILL_INPUT, "lnA and Ea must not be NULL");
    double *rp = reinterpret_cast<double *>(ctx->blob.data() + ctx->off.rpar);
    for (int j = 0; j < ctx->off.M; ++j) {
        if (!std::isfinite(host_lnA[j]) || !std::isfinite(host_Ea[j]))
            return fail(ctx, SUNB_ILL_INPUT, "Arrhenius parameters must be finite");
        rp[3 * j] = host_lnA[j];
        rp[3 * j + 2] = host_Ea[j] / RC;
    }
    CU(cudaMemcpyAsync(ctx->d_tab + ctx->off.rpar, rp, 8 * 3 * ctx->off.M, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->replayed = false;
    return SUNB_SUCCESS;
}


int sunb_graph_capture(sunb_ctx *ctx, double *dev_y, double t0, double dt, int32_t nsteps,
                       int32_t *dev_status)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!dev_y || nsteps < 1 || nsteps > 4096 || !(dt > 0.0) || !std::isfinite(t0))
        return fail(ctx, SUNB_ILL_INPUT, "graph: need y, 1 <= nsteps <= 4096, dt > 0, finite t0");
    if (!ctx->params) return fail(ctx, SUNB_ILL_INPUT, "parameters not set (sunb_set_params)");
    if (ctx->d_tape) return fail(ctx, SUNB_ILL_INPUT, "graph: adjoint-recording contexts integrate one step per call");
    if (ctx->autotune && !ctx->tuned && ctx->tune_cells > 0 && (ctx->kind == SUNB_MECHANISM || ctx->kind == SUNB_MIXED)) {
        const int rc = autotune(ctx, dev_y, t0, t0 + dt);    // the trials synchronise: before building
        if (rc != SUNB_SUCCESS) return rc;
    }
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    ctx->graph_kernels.clear();
    ctx->graph_specs.clear();
    ctx->graph_step.clear();
    CU(cudaGraphCreate(&ctx->graph, 0));
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < nsteps; ++k) {
        const double a = t0 + k * dt, b = t0 + (k + 1) * dt;
        LaunchSpec sp[2];
        int n = 0;
        int rc = step_config(ctx, dev_y, a, b, dev_status, sp, n);
        if (rc != SUNB_SUCCESS) return rc;
        cudaMemsetParams mp{};
        mp.dst = ctx->d_queue;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 8;              // the four 64-bit cell counters
        mp.height = 1;
        mp.pitch = 0;
        cudaGraphNode_t mnode;
        CU(cudaGraphAddMemsetNode(&mnode, ctx->graph, prev ? &prev : nullptr, prev ? 1 : 0, &mp));
        prev = mnode;
        for (int i = 0; i < n; ++i) {
            ctx->graph_specs.push_back(sp[i]);
            ctx->graph_step.push_back(k);
            LaunchSpec &g = ctx->graph_specs.back();
            cudaKernelNodeParams kp{};
            kp.func = g.func;
            kp.gridDim = g.grid;
            kp.blockDim = g.block;
            kp.sharedMemBytes = g.smem;
            void *args[] = {g.arg()};
            kp.kernelParams = args;
            cudaGraphNode_t node;
            CU(cudaGraphAddKernelNode(&node, ctx->graph, &prev, 1, &kp));
            ctx->graph_kernels.push_back(node);
            prev = node;
        }
    }
    CU(cudaGraphInstantiate(&ctx->graph_exec, ctx->graph, 0));
    ctx->graph_dt = dt;
    return SUNB_SUCCESS;
}

int sunb_graph_launch(sunb_ctx *ctx, double t0)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!ctx->graph_exec) return fail(ctx, SUNB_ILL_INPUT, "no captured graph (sunb_graph_capture)");
    if (!std::isfinite(t0)) return fail(ctx, SUNB_ILL_INPUT, "t0 must be finite");
    for (size_t k = 0; k < ctx->graph_kernels.size(); ++k) {
        LaunchSpec &g = ctx->graph_specs[k];
        Controls &c = g.thread ? g.ta.ctl : g.ma.ctl;
        c.t0 = t0 + (double)ctx->graph_step[k] * ctx->graph_dt;
        c.tout = t0 + (double)(ctx->graph_step[k] + 1) * ctx->graph_dt;
        cudaKernelNodeParams kp{};
        kp.func = g.func;
        kp.gridDim = g.grid;
        kp.blockDim = g.block;
        kp.sharedMemBytes = g.smem;
        void *args[] = {g.arg()};
        kp.kernelParams = args;
        CU(cudaGraphExecKernelNodeSetParams(ctx->graph_exec, ctx->graph_kernels[k], &kp));
    }
    CU(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->launches += (int64_t)ctx->graph_kernels.size();
    return SUNB_SUCCESS;
}

int64_t sunb_tape_stride(const sunb_ctx *ctx) { return ctx && ctx->d_tape ? ctx->tape_stride : 0; }

int sunb_get_tapes(sunb_ctx *ctx, int64_t first_cell, int64_t n_cells, double *host_out)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (!ctx->d_tape) return fail(ctx, SUNB_NO_RECORD, "context created without record_adjoint");
    if (first_cell < 0 || n_cells < 0 || first_cell + n_cells > ctx->C || (n_cells > 0 && !host_out))
        return fail(ctx, SUNB_ILL_INPUT, "tapes: need 0 <= first_cell, first_cell + n_cells <= cells, host_out");
    if (n_cells == 0) return SUNB_SUCCESS;
    CU(cudaMemcpyAsync(host_out, ctx->d_tape + first_cell * ctx->tape_stride,
                       8 * (size_t)n_cells * ctx->tape_stride, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return SUNB_SUCCESS;
}

int sunb_get_lanes_per_cell(const sunb_ctx *ctx) { return ctx ? ctx->L : 0; }

int sunb_get_mapping(const sunb_ctx *ctx, int32_t *lanes_per_cell, int32_t *cells_per_cta,
                     int32_t *ctas_per_sm, float *trial_ms)
{
    if (!ctx) return SUNB_ILL_INPUT;
    if (lanes_per_cell) *lanes_per_cell = ctx->L;
    if (cells_per_cta) *cells_per_cta = ctx->cells_per_cta;
    if (ctas_per_sm) *ctas_per_sm = ctx->ctas_per_sm;
    if (trial_ms)
        for (int i = 0; i < 6; ++i) trial_ms[i] = ctx->tune_ms[i / 2][i % 2];
    return SUNB_SUCCESS;
}

int64_t sunb_get_launch_count(const sunb_ctx *ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
