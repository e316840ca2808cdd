// Persistent solve and batch kernels of the FP64 method, templated on PC:
// PC = true builds the engine with its ILU(0) preconditioner passes, PC =
// false without them (no call to them anywhere in the kernel, so the
// unpreconditioned kernels keep their register allocation).  Included by
// mlb_kernels.cu (PC = false, and the dispatch) and mlb_kernels_ilu.cu
// (PC = true), which compile in parallel.
#pragma once

#include <new>

#include "mlb_internal.h"
#include "mlb_refine.cuh"

namespace mlb {

// ===========================================================================
// persistent solve kernel
// ===========================================================================
// One solve by the team described by `gs`: repeated calls of the method
// from the current x while the recursive residual met tol but the true
// residual did not (restart rule of this library), all iterations counted
// against one maxit; then the true residual; the team's rank-0 CTA writes
// the result record.
template <typename T, bool PC, int EW>
__device__ void run_fp64_solve(Engine<T, PC, EW> &E, GridSync &gs, const SolveCtl &ctl, Acct &acct, DevResult *res) {
    using S = typename coef_of<T>::type;
    int64_t total = 0;
    int outer = 0;
    typename Engine<T, PC, EW>::Out o{1, 0, 0, 0, 0.0};
    // ILU(0): the method iterates on y = M x (y_0 = M x_0; x = M^{-1} y at
    // the end, from the final residual pass, which forms M^{-1} y)
    if constexpr (PC) {
        if (E.sys.ilu.lu) E.ilu_to_y();
    }
    for (;;) {
        if (!gs.ok) break;
        o = E.inner(ctl.maxit - total, outer == 0, ctl.tol);
        if (!gs.ok) break;
        total += o.iter;
        if (o.flag != 0 || o.iter == 0 || total >= ctl.maxit || outer >= ctl.max_outer) break;
        outer++;
    }
    int64_t ops_last[5];
    for (int q = 0; q < 5; ++q) ops_last[q] = acct.ops[q];
    double true_rel = __longlong_as_double(0x7ff8000000000000LL);
    if (gs.ok) {
        double bb, rr;
        S qr;
        if (E.ilu_pre(E.sys.x) && E.ph_residual(bb, rr, qr, false)) {
            double bn = sqrt(bb);
            if (bn == 0.0) bn = 1.0;
            true_rel = sqrt(rr) / bn;
            if constexpr (PC) {
                if (E.sys.ilu.lu) E.ilu_to_x();
            }
        }
    }
    if (gs.bid == 0 && threadIdx.x == 0) {
        res->flag = o.flag;
        res->j = o.j;
        res->i = o.i;
        res->status = gs.ok ? 0 : (gs.bar ? ld_relaxed_i32(&gs.bar->status) : kStatusTimeout);
        if (!gs.ok && res->status == 0) res->status = kStatusTimeout;
        res->iter = total;
        res->spmv = acct.spmv;
        res->outer = outer;
        res->err = o.err;
        res->true_relres = true_rel;
        res->bytes = (double)acct.bytes;
        res->flops = (double)acct.flops;
        for (int q = 0; q < 5; ++q) res->ops[q] = ops_last[q];
        res->ctas = (int32_t)gs.nblocks;
    }
}

// Raw shared storage for an object constructed in place by thread 0
// (per-CTA state shared by all threads of the CTA).
template <typename X>
struct alignas(16) SharedSlot {
    unsigned char raw[sizeof(X)];
    __device__ X *get() { return reinterpret_cast<X *>(raw); }
};

// Allow the ring's dynamic shared memory for a kernel (idempotent).
static cudaError_t allow_ring(const void *fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
}

__device__ __forceinline__ void acct_reset(Acct &acct) {
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q) acct.ops[q] = 0;
        acct.spmv = 0;
        acct.bytes = 0;
        acct.flops = 0;
    }
    __syncthreads();
}

template <typename T, bool PC, int EW = 1>
__global__ void __launch_bounds__(kThreads, 1) solve_kernel(SysView<T> sys, SolveCtl ctl) {
    using S = typename coef_of<T>::type;
    extern __shared__ unsigned char dsm[];
    __shared__ double red[kRedDoubles];
    __shared__ S cbuf[kMaxN];
    __shared__ S btbuf[kMaxN];
    __shared__ int sflag;
    __shared__ Acct acct;
    __shared__ TileRing ring;
    __shared__ SysView<T> s_sys;
    __shared__ SolveCtl s_ctl;
    __shared__ SharedSlot<GridSync> gs_slot;
    __shared__ SharedSlot<Engine<T, PC, EW>> e_slot;
    __shared__ unsigned seqs[kThreads];
    ring_init(&ring, ring_buffer(dsm));
    seqs[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_sys = sys;
        s_ctl = ctl;
        new (gs_slot.get()) GridSync(ctl.bar, ctl.partials, red, &sflag, ctl.timeout_ns, &ring, seqs);
        new (e_slot.get()) Engine<T, PC, EW>(s_sys, s_ctl, *gs_slot.get(), cbuf, btbuf, &acct);
    }
    acct_reset(acct);   // includes the __syncthreads that publishes the objects
    GridSync &gs = *gs_slot.get();
    Engine<T, PC, EW> &E = *e_slot.get();
    E.attach();
    run_fp64_solve(E, gs, s_ctl, acct, s_ctl.res);
    __syncthreads();
    ring_drain(&ring, seqs[kConsumers], seqs[0], s_ctl.timeout_ns);
}

// ===========================================================================
// batch: many independent systems in one persistent launch
// ===========================================================================
// Work distribution of a batch launch (BatchPlan).  team_next: the team's
// next position in order_big, agreed on by the team's CTAs: the rank-0 CTA
// takes it from the queue into one of two slots (a slot is rewritten two
// turns later, after every CTA of the team has passed the turn between),
// and a team barrier publishes it.  -1 when order_big is exhausted or the
// barrier failed.
__device__ __forceinline__ int team_next(const BatchPlan &p, unsigned team, unsigned rank, unsigned &tepoch,
                                         unsigned turn, int *sflag, int *s_next) {
    int *slot = p.team_item + 2 * team + (turn & 1u);
    if (rank == 0 && threadIdx.x == 0) *(volatile int *)slot = (int)atomicAdd(&p.queue[1], 1u);
    if (!grid_barrier(p.tbar + team, tepoch, (unsigned)p.team, p.timeout_ns, sflag)) return -1;
    if (threadIdx.x == 0) *s_next = ld_relaxed_i32(slot);
    __syncthreads();
    const int q = *s_next;
    return q < p.count_big ? q : -1;
}

// Runs the plan: solve(item index, team size, rank, barrier, partials) for
// each system this CTA takes (team size 1: this CTA alone).
template <typename Solve>
__device__ __forceinline__ void run_batch_plan(const BatchPlan &p, int *sflag, int *s_next, Solve solve) {
    if (blockIdx.x < (unsigned)(p.teams * p.team)) {
        const unsigned team = blockIdx.x / p.team, rank = blockIdx.x % p.team;
        unsigned tepoch = 0;
        for (unsigned turn = 0;; ++turn) {
            const int q = team_next(p, team, rank, tepoch, turn, sflag, s_next);
            if (q < 0) break;
            solve(p.order_big[q], (unsigned)p.team, rank, p.sbar + q,
                  p.spart + (size_t)q * 2 * kMaxSums * p.team);
        }
    }
    for (;;) {
        if (threadIdx.x == 0) *s_next = (int)atomicAdd(&p.queue[0], 1u);
        __syncthreads();
        const int q = *s_next;
        if (q >= p.count_small) break;
        solve(p.order_small[q], 1u, 0u, (BarrierState *)nullptr, (double *)nullptr);
    }
}

// Each system is solved by the same method as a single solve: by a team
// (the same arithmetic as a solve with grid = team) or by one CTA alone
// with CTA-wide barriers and reductions in shared memory.
template <typename T, bool PC>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(const BatchItem<T> *items, BatchPlan plan) {
    using S = typename coef_of<T>::type;
    extern __shared__ unsigned char dsm[];
    __shared__ TileRing ring;
    __shared__ double red[kRedDoubles];
    __shared__ S cbuf[kMaxN];
    __shared__ S btbuf[kMaxN];
    __shared__ int sflag;
    __shared__ Acct acct;
    __shared__ int s_next;
    __shared__ BatchItem<T> item;
    __shared__ SharedSlot<GridSync> gs_slot;
    __shared__ SharedSlot<Engine<T, PC>> e_slot;
    __shared__ unsigned seqs[kThreads];   // tile counters, kept across systems
    ring_init(&ring, ring_buffer(dsm));
    seqs[threadIdx.x] = 0;
    uint64_t timeout = plan.timeout_ns;
    run_batch_plan(plan, &sflag, &s_next, [&](int idx, unsigned nb, unsigned rk, BarrierState *bar, double *part) {
        if (threadIdx.x == 0) item = items[idx];
        acct_reset(acct);   // includes the __syncthreads that publishes `item`
        timeout = item.ctl.timeout_ns;
        if (threadIdx.x == 0) {
            GridSync *g = nb > 1 ? new (gs_slot.get()) GridSync(bar, part, nb, rk, red, &sflag, timeout, &ring, seqs)
                                 : new (gs_slot.get()) GridSync(red, &sflag, timeout, &ring, seqs);
            new (e_slot.get()) Engine<T, PC>(item.sys, item.ctl, *g, cbuf, btbuf, &acct);
        }
        __syncthreads();
        GridSync &gs = *gs_slot.get();
        Engine<T, PC> &E = *e_slot.get();
        E.attach();
        run_fp64_solve(E, gs, item.ctl, acct, item.ctl.res);
        __syncthreads();
    });
    ring_drain(&ring, seqs[kConsumers], seqs[0], timeout);
}

template <typename T, bool PC>
cudaError_t launch_batch_pc(const BatchItem<T> *items, const BatchPlan &plan, int grid, cudaStream_t st) {
    cudaError_t e = allow_ring((const void *)batch_kernel<T, PC>);
    if (e != cudaSuccess) return e;
    const BatchItem<T> *it = items;
    BatchPlan p = plan;
    void *args[] = {(void *)&it, (void *)&p};
    if (plan.teams > 0)
        return cudaLaunchCooperativeKernel((const void *)batch_kernel<T, PC>, dim3(grid), dim3(kThreads), args,
                                           kRingBytes, st);
    return cudaLaunchKernel((const void *)batch_kernel<T, PC>, dim3(grid), dim3(kThreads), args, kRingBytes, st);
}

template <typename T, bool PC>
int batch_blocks_per_sm_pc() {
    int nb = 0;
    if (allow_ring((const void *)batch_kernel<T, PC>) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<T, PC>, kThreads, kRingBytes) != cudaSuccess)
        return 0;
    return nb;
}

template <typename T, bool PC, int EW = 1>
cudaError_t launch_solve_pc(const SysView<T> &sys, const SolveCtl &ctl, int grid, cudaStream_t st) {
    SysView<T> s = sys;
    SolveCtl c = ctl;
    void *args[] = {(void *)&s, (void *)&c};
    cudaError_t e = allow_ring((const void *)solve_kernel<T, PC, EW>);
    if (e != cudaSuccess) return e;
    if (grid <= 1)
        return cudaLaunchKernel((const void *)solve_kernel<T, PC, EW>, dim3(1), dim3(kThreads), args, kRingBytes,
                                st);
    return cudaLaunchCooperativeKernel((const void *)solve_kernel<T, PC, EW>, dim3(grid), dim3(kThreads), args,
                                       kRingBytes, st);
}

template <typename T, bool PC, int EW = 1>
int solve_blocks_per_sm_pc() {
    int nb = 0;
    if (allow_ring((const void *)solve_kernel<T, PC, EW>) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<T, PC, EW>, kThreads, kRingBytes) !=
            cudaSuccess)
        return 0;
    return nb;
}

// ===========================================================================
// FP32-inner / FP64-refined persistent solve and batch kernels
// ===========================================================================
template <typename T32, typename T64, bool PC>
__global__ void __launch_bounds__(kThreads, 1)
    batch_refine_kernel(const BatchItemR<T32, T64> *items, BatchPlan plan) {
    using S = typename coef_of<T32>::type;
    extern __shared__ unsigned char dsm[];
    __shared__ TileRing ring;
    __shared__ double red[kRedDoubles];
    __shared__ S cbuf[kMaxN];
    __shared__ S btbuf[kMaxN];
    __shared__ int sflag;
    __shared__ Acct acct;
    __shared__ int s_next;
    __shared__ BatchItemR<T32, T64> item;
    __shared__ SharedSlot<GridSync> gs_slot;
    __shared__ SharedSlot<Engine<T32, PC>> e_slot;
    __shared__ SharedSlot<Refiner<T64, T32>> r_slot;
    __shared__ unsigned seqs[kThreads];   // tile counters, kept across systems
    ring_init(&ring, ring_buffer(dsm));
    seqs[threadIdx.x] = 0;
    uint64_t timeout = plan.timeout_ns;
    run_batch_plan(plan, &sflag, &s_next, [&](int idx, unsigned nb, unsigned rk, BarrierState *bar, double *part) {
        if (threadIdx.x == 0) item = items[idx];
        acct_reset(acct);
        timeout = item.ctl.timeout_ns;
        if (threadIdx.x == 0) {
            GridSync *g = nb > 1 ? new (gs_slot.get()) GridSync(bar, part, nb, rk, red, &sflag, timeout, &ring, seqs)
                                 : new (gs_slot.get()) GridSync(red, &sflag, timeout, &ring, seqs);
            new (e_slot.get()) Engine<T32, PC>(item.sys, item.ctl, *g, cbuf, btbuf, &acct);
            new (r_slot.get()) Refiner<T64, T32>(item.rv, *g, &acct);
        }
        __syncthreads();
        GridSync &gs = *gs_slot.get();
        Engine<T32, PC> &E = *e_slot.get();
        Refiner<T64, T32> &R = *r_slot.get();
        E.attach();
        RefineOut o = refine_solve<T32, T64, PC>(E, R, item.ctl, item.rc);
        __syncthreads();
        if (gs.bid == 0 && threadIdx.x == 0) {
            DevResult *res = item.ctl.res;
            res->flag = o.flag;
            res->j = 0;
            res->i = 0;
            res->status = gs.ok ? 0 : (gs.bar ? ld_relaxed_i32(&gs.bar->status) : kStatusTimeout);
            if (!gs.ok && res->status == 0) res->status = kStatusTimeout;
            res->iter = o.iter;
            res->spmv = acct.spmv;
            res->outer = o.outer;
            res->err = o.err;
            res->true_relres = o.err;
            res->bytes = (double)acct.bytes;
            res->flops = (double)acct.flops;
            for (int k = 0; k < 5; ++k) res->ops[k] = acct.ops[k];
            res->ctas = (int32_t)nb;
        }
        __syncthreads();
    });
    ring_drain(&ring, seqs[kConsumers], seqs[0], timeout);
}

template <typename T32, typename T64, bool PC>
cudaError_t launch_batch_refine_pc(const BatchItemR<T32, T64> *items, const BatchPlan &plan, int grid,
                                   cudaStream_t st) {
    cudaError_t e = allow_ring((const void *)batch_refine_kernel<T32, T64, PC>);
    if (e != cudaSuccess) return e;
    const BatchItemR<T32, T64> *it = items;
    BatchPlan p = plan;
    void *args[] = {(void *)&it, (void *)&p};
    if (plan.teams > 0)
        return cudaLaunchCooperativeKernel((const void *)batch_refine_kernel<T32, T64, PC>, dim3(grid),
                                           dim3(kThreads), args, kRingBytes, st);
    return cudaLaunchKernel((const void *)batch_refine_kernel<T32, T64, PC>, dim3(grid), dim3(kThreads), args,
                            kRingBytes, st);
}

template <typename T32, typename T64, bool PC>
int batch_refine_blocks_per_sm_pc() {
    int nb = 0;
    if (allow_ring((const void *)batch_refine_kernel<T32, T64, PC>) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_refine_kernel<T32, T64, PC>, kThreads, kRingBytes) !=
            cudaSuccess)
        return 0;
    return nb;
}

// ===========================================================================
// FP32-inner / FP64-refined persistent solve kernel
// ===========================================================================
template <typename T32, typename T64, bool PC, int EW = 1>
__global__ void __launch_bounds__(kThreads, 1)
    refine_kernel(SysView<T32> sys, RefView<T64> rv, SolveCtl ctl, RefCtl rc) {
    using S = typename coef_of<T32>::type;
    extern __shared__ unsigned char dsm[];
    __shared__ TileRing ring;
    __shared__ double red[kRedDoubles];
    __shared__ S cbuf[kMaxN];
    __shared__ S btbuf[kMaxN];
    __shared__ int sflag;
    __shared__ Acct acct;
    __shared__ SysView<T32> s_sys;
    __shared__ RefView<T64> s_rv;
    __shared__ SolveCtl s_ctl;
    __shared__ RefCtl s_rc;
    __shared__ SharedSlot<GridSync> gs_slot;
    __shared__ SharedSlot<Engine<T32, PC, EW>> e_slot;
    __shared__ SharedSlot<Refiner<T64, T32, EW>> r_slot;
    __shared__ unsigned seqs[kThreads];
    ring_init(&ring, ring_buffer(dsm));
    seqs[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_sys = sys;
        s_rv = rv;
        s_ctl = ctl;
        s_rc = rc;
        GridSync *g = new (gs_slot.get()) GridSync(ctl.bar, ctl.partials, red, &sflag, ctl.timeout_ns, &ring, seqs);
        new (e_slot.get()) Engine<T32, PC, EW>(s_sys, s_ctl, *g, cbuf, btbuf, &acct);
        new (r_slot.get()) Refiner<T64, T32, EW>(s_rv, *g, &acct);
    }
    acct_reset(acct);   // includes the __syncthreads that publishes the objects
    GridSync &gs = *gs_slot.get();
    Engine<T32, PC, EW> &E = *e_slot.get();
    Refiner<T64, T32, EW> &R = *r_slot.get();
    E.attach();
    RefineOut o = refine_solve<T32, T64, PC, EW>(E, R, s_ctl, s_rc);
    __syncthreads();
    ring_drain(&ring, seqs[kConsumers], seqs[0], ctl.timeout_ns);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevResult *res = ctl.res;
        res->flag = o.flag;
        res->j = 0;
        res->i = 0;
        res->status = gs.ok ? 0 : ld_relaxed_i32(&ctl.bar->status);
        if (!gs.ok && res->status == 0) res->status = kStatusTimeout;
        res->iter = o.iter;
        res->spmv = acct.spmv;
        res->outer = o.outer;
        res->err = o.err;
        res->true_relres = o.err;
        res->bytes = (double)acct.bytes;
        res->flops = (double)acct.flops;
        for (int q = 0; q < 5; ++q) res->ops[q] = acct.ops[q];
        res->ctas = (int32_t)gridDim.x;
    }
}

template <typename T32, typename T64, bool PC, int EW = 1>
cudaError_t launch_refine_pc(const SysView<T32> &sys, const RefView<T64> &rv, const SolveCtl &ctl,
                          const RefCtl &rc, int grid, cudaStream_t st) {
    SysView<T32> s = sys;
    RefView<T64> r = rv;
    SolveCtl c = ctl;
    RefCtl q = rc;
    void *args[] = {(void *)&s, (void *)&r, (void *)&c, (void *)&q};
    cudaError_t e = allow_ring((const void *)refine_kernel<T32, T64, PC, EW>);
    if (e != cudaSuccess) return e;
    if (grid <= 1)
        return cudaLaunchKernel((const void *)refine_kernel<T32, T64, PC, EW>, dim3(1), dim3(kThreads), args, kRingBytes,
                                st);
    return cudaLaunchCooperativeKernel((const void *)refine_kernel<T32, T64, PC, EW>, dim3(grid), dim3(kThreads),
                                       args, kRingBytes, st);
}

template <typename T32, typename T64, bool PC, int EW = 1>
int refine_blocks_per_sm_pc() {
    int nb = 0;
    if (allow_ring((const void *)refine_kernel<T32, T64, PC, EW>) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, refine_kernel<T32, T64, PC, EW>, kThreads, kRingBytes) !=
            cudaSuccess)
        return 0;
    return nb;
}

// 3x3-block storage (real values only), instantiated in mlb_kernels_bsr.cu.
extern template cudaError_t launch_solve_pc<double, false, 3>(const SysView<double> &, const SolveCtl &, int,
                                                              cudaStream_t);
extern template cudaError_t launch_solve_pc<double, true, 3>(const SysView<double> &, const SolveCtl &, int,
                                                             cudaStream_t);
extern template int solve_blocks_per_sm_pc<double, false, 3>();
extern template int solve_blocks_per_sm_pc<double, true, 3>();
extern template cudaError_t launch_refine_pc<float, double, false, 3>(const SysView<float> &,
                                                                      const RefView<double> &, const SolveCtl &,
                                                                      const RefCtl &, int, cudaStream_t);
extern template cudaError_t launch_refine_pc<float, double, true, 3>(const SysView<float> &,
                                                                     const RefView<double> &, const SolveCtl &,
                                                                     const RefCtl &, int, cudaStream_t);
extern template int refine_blocks_per_sm_pc<float, double, false, 3>();
extern template int refine_blocks_per_sm_pc<float, double, true, 3>();

// Instantiated in mlb_kernels_ilu.cu.
extern template cudaError_t launch_refine_pc<float, double, true>(const SysView<float> &, const RefView<double> &,
                                                                  const SolveCtl &, const RefCtl &, int,
                                                                  cudaStream_t);
extern template cudaError_t launch_refine_pc<cfloat, cdouble, true>(const SysView<cfloat> &,
                                                                    const RefView<cdouble> &, const SolveCtl &,
                                                                    const RefCtl &, int, cudaStream_t);
extern template int refine_blocks_per_sm_pc<float, double, true>();
extern template int refine_blocks_per_sm_pc<cfloat, cdouble, true>();
extern template cudaError_t launch_batch_refine_pc<float, double, true>(const BatchItemR<float, double> *,
                                                                        const BatchPlan &, int, cudaStream_t);
extern template cudaError_t launch_batch_refine_pc<cfloat, cdouble, true>(const BatchItemR<cfloat, cdouble> *,
                                                                          const BatchPlan &, int, cudaStream_t);
extern template int batch_refine_blocks_per_sm_pc<float, double, true>();
extern template int batch_refine_blocks_per_sm_pc<cfloat, cdouble, true>();

// Instantiated in mlb_kernels_cplx.cu.
extern template cudaError_t launch_solve_pc<cdouble, false>(const SysView<cdouble> &, const SolveCtl &, int,
                                                            cudaStream_t);
extern template int solve_blocks_per_sm_pc<cdouble, false>();
extern template cudaError_t launch_batch_pc<cdouble, false>(const BatchItem<cdouble> *, const BatchPlan &, int,
                                                            cudaStream_t);
extern template int batch_blocks_per_sm_pc<cdouble, false>();

extern template cudaError_t launch_solve_pc<double, true>(const SysView<double> &, const SolveCtl &, int, cudaStream_t);
extern template cudaError_t launch_solve_pc<cdouble, true>(const SysView<cdouble> &, const SolveCtl &, int,
                                                          cudaStream_t);
extern template cudaError_t launch_batch_pc<double, true>(const BatchItem<double> *, const BatchPlan &, int,
                                                         cudaStream_t);
extern template cudaError_t launch_batch_pc<cdouble, true>(const BatchItem<cdouble> *, const BatchPlan &, int,
                                                          cudaStream_t);
extern template int solve_blocks_per_sm_pc<double, true>();
extern template int solve_blocks_per_sm_pc<cdouble, true>();
extern template int batch_blocks_per_sm_pc<double, true>();
extern template int batch_blocks_per_sm_pc<cdouble, true>();

}  // namespace mlb
