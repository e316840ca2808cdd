// FP32-inner / FP64-refined solve: the outer FP64 iterative refinement
// around the FP32 ML(n)BiCGStab engine, in the same persistent kernel.
//
//   repeat:  r = b - A x                       (FP64 SpMV, ||b||, ||r||)
//            stop when ||r||/||b|| < tol
//            solve A d = r / ||r|| in FP32      (ML(n)BiCGStabt, x_0 = 0,
//                                                relative tolerance inner_tol)
//            x = x + ||r|| d                    (FP64)
//
// The inner right-hand side is scaled to unit norm so that FP32 never sees
// the shrinking magnitudes of later residuals.  All recurrence coefficients
// of the inner method are FP64 scalars; its vectors, matrix values and
// per-thread accumulations are FP32.
#pragma once

#include "mlb_engine.cuh"

namespace mlb {

// FP64 side of a refined solve.
template <typename T64>
struct RefView {
    int64_t N, ld, nnz, nslices;
    const int64_t *slice_ptr;
    const int32_t *scol;
    const T64 *sval;   // FP64 values, same SELL-32 layout as the FP32 copy
    int spt[3];        // slices per SpMV tile for FP64 values, 0/1/2 epilogue vectors
    T64 *x;            // solution
    const T64 *b;
    T64 *r;            // true residual
};

struct RefCtl {
    double inner_tol;
    int64_t inner_maxit;
};

template <typename T64, typename T32>
struct Refiner {
    using ACC = double;
    static constexpr int DS = dslots<T64>();
    const RefView<T64> &v;
    GridSync &gs;
    Acct *acct;
    const T32 *x32;   // inner solution d
    int64_t s_lo, s_hi;   // owned slices (the same rows as the inner engine)

    // Constructed by one thread in shared memory, like the engine.
    __device__ Refiner(const RefView<T64> &v_, GridSync &g, Acct *a, const T32 *x32_)
        : v(v_), gs(g), acct(a), x32(x32_) {
        own_range(v_.nslices, g.nblocks, g.bid, s_lo, s_hi);
    }

    // r = b - A x in FP64; sums ||b||^2, ||r||^2.
    __device__ __noinline__ bool residual(double &bb, double &rr) {
        double acc[2] = {0.0, 0.0};
        const T64 *epi[1] = {v.b};
        T64 *const r = v.r;
        unsigned sq = gs.seq();   // issued (producer lane) or consumed (consumers) tiles
        bool okt = sell_spmv<1>(gs.ring, sq, sq, gs.timeout_ns, s_lo, s_hi, v.spt[1], v.slice_ptr, v.scol, v.sval,
                                v.x, epi, threadIdx.x & 31,
                                [=](int64_t row, T64 y, const T64 (&e)[1], double(&a)[2]) {
                                    T64 rv = subT(e[0], y);
                                    r[row] = rv;
                                    acc_nrm(&a[0], e[0]);
                                    acc_nrm(&a[1], rv);
                                },
                                acc);
        gs.seq() = sq;
        if (!okt) gs.ring->failed = 1;
        if (!gs.template reduce<2>(acc)) return false;
        if (gs.ring->failed) { gs.ok = false; return false; }
        bb = acc[0];
        rr = acc[1];
        if (threadIdx.x == 0) {
            acct->bytes += (double)v.nnz * (sizeof(T64) + 4) + 4.0 * (double)(v.N + 1) +
                           3.0 * (double)v.N * sizeof(T64);
            acct->spmv++;
        }
        return true;
    }

    // x += scale * d (d from the FP32 inner solve).  Chunks of 16 bytes of
    // the FP32 vector, i.e. 32 bytes of the FP64 one.
    __device__ __noinline__ bool update(double scale) {
        constexpr int PW = Pack<T32>::W;
        static_assert(PW * sizeof(T64) == 32, "an FP32 chunk maps to two FP64 chunks");
        constexpr int CPS = 32 * sizeof(T32) / 16;   // FP32 chunks per slice
        const int64_t c_hi = s_hi * CPS;
        const int64_t c_start = s_lo * CPS + ((threadIdx.x >> 5) < kConsumerWarps ? threadIdx.x : c_hi);
        const T32 *const d32 = x32;
        T64 *const x64 = v.x;
        for (int64_t ch = c_start; ch < c_hi; ch += kConsumers) {
            Pack<T32> d = ldp(d32, ch);
            uint4 *xp = reinterpret_cast<uint4 *>(x64) + 2 * ch;
            uint4 w2[2] = {xp[0], xp[1]};
            T64 xv[PW];
            memcpy(xv, w2, sizeof(xv));
#pragma unroll
            for (int e = 0; e < PW; ++e) xv[e] = widen_fma(scale, d.e[e], xv[e]);
            memcpy(w2, xv, sizeof(xv));
            xp[0] = w2[0];
            xp[1] = w2[1];
        }
        fence_proxy_async_global();
        if (threadIdx.x == 0) acct->bytes += (double)v.N * (2.0 * sizeof(T64) + sizeof(T32));
        return gs.sync();
    }

    __device__ __forceinline__ static double widen_fma(double s, float d, double x) { return fma(s, (double)d, x); }
    __device__ __forceinline__ static cdouble widen_fma(double s, cfloat d, cdouble x) {
        return {fma(s, (double)d.re, x.re), fma(s, (double)d.im, x.im)};
    }
};

struct RefineOut {
    int flag;
    int64_t iter;
    int outer;
    double err;
};

// Outer refinement loop (see the file comment).  `rec` records the true
// relative residual of every outer step in ctl.err_hist.
template <typename T32, typename T64>
__device__ RefineOut refine_solve(Engine<T32> &E, Refiner<T64, T32> &R, const SolveCtl &ctl, const RefCtl &rc) {
    RefineOut out{1, 0, 0, __longlong_as_double(0x7ff8000000000000LL)};
    double prev = 0.0;
    int stalled = 0;
    for (;;) {
        double bb, rr;
        if (!R.residual(bb, rr)) return out;
        double bn = sqrt(bb);
        if (bn == 0.0) bn = 1.0;
        const double rn = sqrt(rr);
        const double err = rn / bn;
        out.err = err;
        if (ctl.err_hist && out.outer < ctl.hist_cap && E.gs.bid == 0 && threadIdx.x == 0)
            ctl.err_hist[out.outer] = err;
        if (err < ctl.tol) { out.flag = 0; return out; }
        if (!(err == err)) { out.flag = -1; return out; }
        if (out.outer >= ctl.max_outer || out.iter >= ctl.maxit) { out.flag = 1; return out; }
        if (out.outer > 0 && err > 0.99 * prev) {
            if (++stalled >= 2) { out.flag = 1; return out; }
        } else {
            stalled = 0;
        }
        prev = err;
        int64_t budget = ctl.maxit - out.iter;
        if (budget > rc.inner_maxit) budget = rc.inner_maxit;
        const double scale = rn > 0.0 ? 1.0 / rn : 1.0;
        auto o = E.inner(budget, false, rc.inner_tol, R.v.r, scale);
        if (!E.gs.ok) return out;
        out.iter += o.iter;
        if (o.flag == -1 && o.iter == 0) { out.flag = -1; return out; }
        if (!R.update(rn)) return out;
        out.outer++;
    }
}

}  // namespace mlb
