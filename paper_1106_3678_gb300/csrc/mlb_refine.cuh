// FP32-inner / FP64-refined solve: ML(n)BiCGStab in FP32 inside an FP64
// iterative refinement, in the same persistent kernel.
//
//   repeat:  r = b - A x                        (FP64 SpMV, ||b||, ||r||)
//            stop when ||r||/||b|| < tol
//            solve A d = r / ||r|| in FP32       (ML(n)BiCGStabt, d_0 = 0)
//            x = x + ||r|| d                     (FP64)
//
// The inner solve keeps its Krylov recurrences across refinement steps
// (residual replacement; reliable updates in the sense of Sleijpen & van
// der Vorst 1996 and van der Vorst & Ye 2000): whenever its recursive
// residual has fallen by a factor `delta` below the largest value since
// the last update (checked at block ends), or has met the tolerance, the
// FP32 iterate d is moved into the FP64 solution (x += ||r|| d, d = 0),
// the FP64 true residual b - A x is formed, and the FP32 residual is
// replaced by it (scaled by the same 1/||r||).  The inner call therefore
// stops only when the true FP64 residual meets tol, and the gap between
// the FP32 recursive residual and the true one never grows beyond what
// one stretch between updates accumulates.
//
// Safeguards: an inner call also ends when its residual has not reached a
// new minimum for max(`window`, iterations it took to reach the current
// minimum) iterations (stagnation) or after `inner_maxit` iterations; the remaining FP32 iterate is then moved into x.  The outer
// loop keeps the solution with the smallest true residual so far (xbest):
// when an inner call ends with a larger one, xbest is returned (flag 1).
// A new inner call restarts from the current x; the solve also stops with
// flag 1 after two inner calls in a row that each left the true residual
// above 0.9 times its value at their start.
//
// All recurrence coefficients of the inner method are FP64 scalars; its
// vectors, matrix values, preconditioner factors and per-thread
// accumulations are FP32.  With a preconditioner the inner solve works on
// A M^{-1} (M = diag(A) stored in the matrix values, or the FP32 ILU(0)
// factors applied by the engine's triangular solves); with ILU(0) its
// iterate is y = M d, so moving it into x first forms d = M^{-1} y.
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
    T64 *xbest;        // the solution with the smallest true residual so far
};

struct RefCtl {
    double delta;         // reliable-update factor (inner_tol of the options)
    int64_t inner_maxit;  // iteration cap of one inner call
    int64_t window;       // stagnation window of one inner call
};

template <typename T64, typename T32, int EW = 1>
struct Refiner {
    using ACC = double;
    static constexpr int DS = dslots<T64>();
    const RefView<T64> &v;
    GridSync &gs;
    Acct *acct;
    int64_t s_lo, s_hi;   // owned slices (the same rows as the inner engine)

    // Constructed by one thread in shared memory, like the engine.
    __device__ Refiner(const RefView<T64> &v_, GridSync &g, Acct *a) : v(v_), gs(g), acct(a) {
        own_range(v_.nslices, g.nblocks, g.bid, s_lo, s_hi);
    }

    // r = b - A x in FP64; sums ||b||^2, ||r||^2.
    __device__ __noinline__ bool residual(double &bb, double &rr) {
        double acc[2] = {0.0, 0.0};
        const T64 *epi[1] = {v.b};
        T64 *const r = v.r;
        unsigned sq = gs.seq();   // issued (producer lane) or consumed (consumers) tiles
        bool okt = sell_spmv<1, EW>(gs.ring, sq, sq, gs.timeout_ns, s_lo, s_hi, v.spt[1], v.slice_ptr, v.scol, v.sval,
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
            acct->bytes += v.nnz * (int64_t)sizeof(T64) + v.nnz / EW * 4 + 4 * (v.N + 1) +
                           3 * v.N * (int64_t)sizeof(T64);
            acct->flops += (DS == 2 ? 8 : 2) * v.nnz + (DS == 2 ? 10 : 5) * v.N;
            acct->spmv++;
        }
        return true;
    }

    // x += scale * d (d from the FP32 inner solve, rows of this CTA; with
    // ILU(0) d = M^{-1} y, written by every CTA of the team, so read
    // through L2), then zero[...] = 0 on the same rows when zero != null.
    // Chunks of 16 bytes of the FP32 vector, i.e. 32 bytes of the FP64 one.
    __device__ __noinline__ bool update(double scale, const T32 *d32, T32 *zero) {
        constexpr int PW = Pack<T32>::W;
        static_assert(PW * sizeof(T64) == 32, "an FP32 chunk maps to two FP64 chunks");
        constexpr int CPS = 32 * sizeof(T32) / 16;   // FP32 chunks per slice
        const int64_t c_hi = s_hi * CPS;
        const int64_t c_start = s_lo * CPS + ((threadIdx.x >> 5) < kConsumerWarps ? threadIdx.x : c_hi);
        T64 *const x64 = v.x;
        for (int64_t ch = c_start; ch < c_hi; ch += kConsumers) {
            Pack<T32> d;
            *reinterpret_cast<uint4 *>(&d) = __ldcg(reinterpret_cast<const uint4 *>(d32) + ch);
            uint4 *xp = reinterpret_cast<uint4 *>(x64) + 2 * ch;
            uint4 w2[2] = {xp[0], xp[1]};
            T64 xv[PW];
            memcpy(xv, w2, sizeof(xv));
#pragma unroll
            for (int e = 0; e < PW; ++e) xv[e] = widen_fma(scale, d.e[e], xv[e]);
            memcpy(w2, xv, sizeof(xv));
            xp[0] = w2[0];
            xp[1] = w2[1];
            if (zero) reinterpret_cast<uint4 *>(zero)[ch] = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_proxy_async_global();
        if (threadIdx.x == 0)
            acct->bytes += v.N * (int64_t)(2 * sizeof(T64) + (zero ? 2 : 1) * sizeof(T32));
        return gs.sync();
    }

    // xbest = x (save) or x = xbest (restore) on the rows of this CTA.
    __device__ __noinline__ bool keep(bool save) {
        constexpr int CPS64 = 32 * sizeof(T64) / 16;   // FP64 chunks per slice
        const int64_t c_hi = s_hi * CPS64;
        const int64_t c_start = s_lo * CPS64 + ((threadIdx.x >> 5) < kConsumerWarps ? threadIdx.x : c_hi);
        uint4 *dst = reinterpret_cast<uint4 *>(save ? v.xbest : v.x);
        const uint4 *src = reinterpret_cast<const uint4 *>(save ? v.x : v.xbest);
        for (int64_t ch = c_start; ch < c_hi; ch += kConsumers) dst[ch] = src[ch];
        if (threadIdx.x == 0) acct->bytes += 2 * v.N * (int64_t)sizeof(T64);
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

// Residual replacement of one inner call (see the file comment and
// Engine::inner).  A per-thread object: every thread holds the same values.
template <typename T32, typename T64, bool PC, int EW = 1>
struct RelUpdate {
    static constexpr bool kActive = true;
    using S = typename coef_of<T32>::type;
    Engine<T32, PC, EW> *E;
    Refiner<T64, T32, EW> *R;
    double sigma;      // ||r|| at the start of the call: the inner system is A d = r / sigma
    double bn;         // ||b||
    double tol;        // target of the true relative residual
    double delta;
    int64_t window;
    double mr;         // largest recursive residual since the last update
    double best;       // smallest residual seen at a block end
    int64_t best_it;
    double true_err;   // true relative residual after the last update
    int updates;

    __device__ void track(double err) { mr = err > mr ? err : mr; }
    __device__ void reset(double err) { mr = err; }
    __device__ bool want(double err) const { return err < delta * mr; }
    // No new smallest residual for `window` iterations, and for at least as
    // many iterations as it took to reach the smallest one (a call that
    // made progress for a long time may sit on a plateau as long).
    __device__ bool stalled(int64_t iter, double err) {
        if (err < best) {
            best = err;
            best_it = iter;
            return false;
        }
        const int64_t w = best_it > window ? best_it : window;
        return iter - best_it > w;
    }
    // The inner iterate into x, the true residual, r replaced (see
    // Engine::inner for the arguments).
    __device__ __noinline__ bool replace(int qcol, bool f0, double &rr, S &qr, S &fr, bool &conv) {
        const T32 *d = E->sys.x;
        if constexpr (PC) {
            if (E->sys.ilu.lu) {
                if (!E->ilu_solve(E->sys.x, E->sys.ilu.t)) return false;
                d = E->sys.ilu.t;
            }
        }
        if (!R->update(sigma, d, E->sys.x)) return false;
        double bb, r64;
        if (!R->residual(bb, r64)) return false;
        true_err = sqrt(r64) / bn;
        conv = true_err < tol;
        if (!E->ph_replace_narrow(R->v.r, 1.0 / sigma, qcol, f0, rr, qr, fr)) return false;
        updates++;
        return true;
    }
};

// Outer refinement loop (see the file comment).  ctl.err_hist records the
// true relative residual at the start of every inner call, and the final
// one.
template <typename T32, typename T64, bool PC, int EW = 1>
__device__ RefineOut refine_solve(Engine<T32, PC, EW> &E, Refiner<T64, T32, EW> &R, const SolveCtl &ctl,
                                  const RefCtl &rc) {
    RefineOut out{1, 0, 0, __longlong_as_double(0x7ff8000000000000LL)};
    double prev = 0.0;   // true residual at the start of the last inner call
    double best = 0.0;   // true residual of the saved solution xbest
    int no_gain = 0;
    auto record = [&](double err) {
        if (ctl.err_hist && out.outer < ctl.hist_cap && E.gs.bid == 0 && threadIdx.x == 0)
            ctl.err_hist[out.outer] = err;
    };
    for (;;) {
        double bb, rr;
        if (!R.residual(bb, rr)) return out;
        double bn = sqrt(bb);
        if (bn == 0.0) bn = 1.0;
        double err = sqrt(rr) / bn;
        if (out.outer > 0 && !(err <= best)) {
            // the last inner call left x worse than the best solution so
            // far: return that one (a new call from it would repeat the
            // same iteration)
            if (!R.keep(false) || !R.residual(bb, rr)) return out;
            out.err = sqrt(rr) / bn;
            record(out.err);
            out.flag = 1;
            return out;
        }
        if (!(err == err)) {
            out.err = err;
            record(err);
            out.flag = -1;
            return out;
        }
        if (!R.keep(true)) return out;
        best = err;
        out.err = err;
        record(err);
        if (err < ctl.tol) { out.flag = 0; return out; }
        if (out.outer >= ctl.max_outer || out.iter >= ctl.maxit) { out.flag = 1; return out; }
        if (out.outer > 0 && !(err <= 0.9 * prev)) {
            if (++no_gain >= 2) { out.flag = 1; return out; }
        } else {
            no_gain = 0;
        }
        prev = err;
        int64_t budget = ctl.maxit - out.iter;
        if (budget > rc.inner_maxit) budget = rc.inner_maxit;
        const double rn = sqrt(rr);
        RelUpdate<T32, T64, PC, EW> hk{&E, &R, rn, bn, ctl.tol, rc.delta, rc.window, 0.0, INFINITY, 0, err, 0};
        auto o = E.inner(budget, false, ctl.tol * bn / rn, R.v.r, 1.0 / rn, &hk);
        if (!E.gs.ok) return out;
        out.iter += o.iter;
        out.outer++;
        if (o.flag == 0) {
            // converged on the true residual at the last update
            out.err = hk.true_err;
            out.flag = 0;
            record(out.err);
            return out;
        }
        if (o.flag == -1 && o.iter == 0) { out.flag = -1; return out; }
        // move what the inner call accumulated since its last update
        const T32 *d = E.sys.x;
        if constexpr (PC) {
            if (E.sys.ilu.lu) {
                if (!E.ilu_solve(E.sys.x, E.sys.ilu.t)) return out;
                d = E.sys.ilu.t;
            }
        }
        if (!R.update(rn, d, nullptr)) return out;
    }
}

}  // namespace mlb
