// Device pieces shared by the translation units of the library: the cell
// queue, the per-cell counters, the cooling-table staging and the
// thread-per-cell kernel.  Both the context entry points (sunb_api.cu) and
// the allocation-free one (sunb_noalloc.cu) launch this same kernel, so a
// cell's arithmetic is identical through either.
#pragma once
#include <cstdint>

#include "sunb_common.cuh"
#include "bdf_control.cuh"
#include "cell_thread.cuh"
#include "erk_control.cuh"

namespace sunb {

// Cell indices handed out by a global counter (the device work queue):
// a finished group or thread takes the next unstarted cell, so cells whose
// step counts differ by orders of magnitude do not leave lanes idle.
__device__ __forceinline__ long long grab_group(unsigned long long *q, int lane, unsigned mask, int L)
{
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(q, 1ull);
    return (long long)__shfl_sync(mask, v, 0, L);
}

__device__ __forceinline__ long long grab_thread(unsigned long long *q)
{
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    const int rank = __popc(m & ((1u << lane) - 1u));
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(q, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    return (long long)(base + rank);
}

__device__ __forceinline__ void write_stats(int32_t *stats, int32_t *status, long long cell,
                                            const CellStats &s)
{
    int4 *p = reinterpret_cast<int4 *>(stats + 8 * cell);
    p[0] = make_int4(s.nst, s.nfe, s.nje, s.nni);
    p[1] = make_int4(s.ncf, s.nef, s.qlast, s.status);
    if (status) status[cell] = s.status;
}

struct CoolArgs {
    const double *knots;   // [3 * n + EXP_TABLE_SIZE]: lnT, lnLam, slope (n-1 used), exp table
    int n;
    double gamma_heat;
};

__device__ __forceinline__ void stage_bytes(unsigned char *dst, const unsigned char *src, int bytes)
{
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// The cooling table in shared memory: lnT, lnLam, slope (n each, the last
// slope unused), the exp table, then lnT rounded to float (the knot search).
__host__ __device__ __forceinline__ int cooling_smem_bytes(int n)
{
    return 8 * (3 * n + EXP_TABLE_SIZE) + 4 * n;
}

__device__ __forceinline__ CoolingSmem stage_cooling(unsigned char *dst, const CoolArgs &c)
{
    double *d = reinterpret_cast<double *>(dst);
    float *df = reinterpret_cast<float *>(d + 3 * c.n + EXP_TABLE_SIZE);
    for (int i = threadIdx.x; i < 3 * c.n + EXP_TABLE_SIZE; i += blockDim.x) d[i] = c.knots[i];
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) df[i] = (float)c.knots[i];
    CoolingSmem t;
    t.n = c.n;
    t.gamma_heat = c.gamma_heat;
    t.lnT = d;
    t.lnLam = d + c.n;
    t.slope = d + 2 * c.n;
    t.exptab = d + 3 * c.n;
    t.lnTf = df;
    return t;
}

struct ThreadArgs {
    long long n;
    double *y;
    const double *params;
    int32_t *stats, *status;
    unsigned long long *queue;
    Controls ctl;
    double atol[3];
    CoolArgs cool;
    int spread_lanes;   // > 0: one wave, lanes [0, spread_lanes) of every warp take a cell each
    double *tape;       // step-history tapes (the REC kernel), tape_stride doubles per cell
    long long tape_stride;
    int tape_cap;
};

// Thread-per-cell kernel for Robertson and cosmology batches.  Large batches
// take cells from the device queue; a batch that fits in one wave
// (spread_lanes > 0) is spread over all SMs and warps instead, cell
// b + grid (w + W l) for lane l < spread_lanes of warp w of CTA b, so that
// few cells do not crowd a few SMs.  ERK: the explicit Runge-Kutta
// controller instead of the BDF one (a separate kernel).  REC: record each
// cell's step history to its tape (a separate kernel).
template <class Prob, bool ERK = false, bool REC = false>
__global__ void __launch_bounds__(256) thread_kernel(const ThreadArgs a)
{
    __shared__ __align__(16) double cool_s[3 * 256 + EXP_TABLE_SIZE + 128];
    CoolingSmem cool;
    if (Prob::N == 1) cool = stage_cooling(reinterpret_cast<unsigned char *>(cool_s), a.cool);
    __syncthreads();
    ThreadCell<Prob, REC> tc;
    if constexpr (Prob::N == 1) tc.prob.tab = &cool;
#pragma unroll
    for (int i = 0; i < Prob::N; ++i) tc.atol[i] = a.atol[i];
    bool taken = false;
    auto next = [&]() -> long long {
        if (a.spread_lanes > 0) {
            const int l = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
            if (taken || l >= a.spread_lanes) return -1;
            taken = true;
            const long long cell = blockIdx.x + (long long)gridDim.x * (w + (long long)W * l);
            return cell < a.n ? cell : -1;
        }
        const long long cell = grab_thread(a.queue);
        return cell < a.n ? cell : -1;
    };
    auto bind = [&](long long cell) {
        tc.prob.load(a.params, cell);
        tc.yg = a.y + cell * Prob::N;
        if constexpr (REC) {
            tc.tape = a.tape + cell * a.tape_stride;
            tc.tape_cap = a.tape_cap;
        }
    };
    auto done = [&](long long cell, const CellStats &st) { write_stats(a.stats, a.status, cell, st); };
    if constexpr (ERK) run_cells<ErkRun>(tc, a.ctl, launched_warp_mask(), next, bind, done);
    else run_cells(tc, a.ctl, launched_warp_mask(), next, bind, done);
}

}  // namespace sunb
