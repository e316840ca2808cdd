// Persistent solve engine: ML(n)BiCGStabt (Algorithm 7.1 with M = I, i.e.
// Algorithm 4.1 with its k-loop split as k = jn + i, eq. 2.1) as one
// kernel launch.
//
// Every step of the method is a "pass" over the rows: a streaming update of
// a few N-vectors fused with the inner product(s) the next step needs, or a
// SELL-32 SpMV fused with its inner products.  Each pass ends in a
// deterministic reduction: per-CTA partial sums, a grid barrier, then every
// CTA sums the partials in the same fixed order.  All scalars (alpha,
// beta~, beta, omega, c, e, err) are therefore bit-identical in every CTA,
// and every CTA takes the same branches (convergence, breakdown, g_n/r_n
// bookkeeping) without any host round trip.
//
// Storage ("ring"): g_k, w_k, c_k of iterate k = jn + s live in slot
// s = k mod n of G, W, c.  During step jn+i, slots < i hold block j and
// slots >= i still hold block j-1, as Algorithm 7.1 reads them.
//
// Fusions (none changes the order of any floating-point operation of a
// single element):
//   * x and r updates (alpha step) fused with ||r||^2, q_{i+1}^H r and, in
//     block 0, f_1^H r.
//   * the z_w sweep over block j-1 (Algorithm 7.1, steps 10-17) makes one
//     pass per coefficient over z_w only; the g-updates of that sweep feed
//     no inner product, so all of them run in the last pass, in the same
//     order, fused with the omega-correction (step 18) and the first
//     f-inner product (step 20).
//   * each f-sweep pass applies one update and computes the next f^H g.
//   * SpMV with the epilogue inner products c = q^H w (step 32), or
//     (A u)^H (A u) and (A u)^H u (step 38).
#pragma once

#include "mlb_device.cuh"

namespace mlb {

constexpr int kThreads = 512;   // threads per CTA of the solve kernels
constexpr int kMaxN = 64;       // largest number of shadow vectors
constexpr int kMaxSums = 8;     // doubles reduced per pass (max)

// Result record written by CTA 0 at the end of a solve.
struct DevResult {
    int32_t flag, j, i, status;
    int64_t iter, spmv, outer;
    double err, true_relres, bytes;
    int64_t ops[5];
};

enum { OP_MATVEC = 0, OP_DOT = 1, OP_SAXPY = 2, OP_SCALE = 3, OP_NORM = 4 };

// Per-CTA accounting in shared memory (identical in every CTA).
struct Acct {
    int64_t ops[5];   // Table 4.3 categories of the current inner call
    int64_t spmv;     // all sparse products of the solve
    double bytes;     // algorithmic bytes of the solve
};

// Device view of one linear system.  Vectors have leading dimension `ld`
// (a multiple of 512 elements); entries N..ld-1 are zero and stay zero.
template <typename T>
struct SysView {
    int64_t N, ld, nnz;
    int64_t nslices;            // ld / 32
    const int64_t *slice_ptr;   // SELL-32: slice s spans [slice_ptr[s], slice_ptr[s+1])
    const int32_t *scol;        // column of entry (slice, k, lane) at off + 32k + lane
    const T *sval;
    const T *Q;                 // ld x n
    const T *F;                 // ld x (n-1), F = A^H Q(:,0:n-2)
    T *G, *W;                   // ld x n rings
    T *x, *r, *z;               // ld
    T *b;                       // ld (written only by the refined-mode inner start)
    int n;
};

struct SolveCtl {
    double tol;
    int64_t maxit;
    double kappa;
    int max_outer;
    double *err_hist;           // device, may be null
    int64_t hist_cap;
    double *partials;           // [2][kMaxSums][gridDim]
    BarrierState *bar;
    DevResult *res;
    uint64_t timeout_ns;
};

// ---- element helpers used by Engine ---------------------------------------
__device__ __forceinline__ double subT(double a, double b) { return a - b; }
__device__ __forceinline__ float subT(float a, float b) { return a - b; }
template <typename R>
__device__ __forceinline__ cx<R> subT(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }

__device__ __forceinline__ double ldg_val(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldg_val(const float *p) { return __ldg(p); }
__device__ __forceinline__ cdouble ldg_val(const cdouble *p) {
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cfloat ldg_val(const cfloat *p) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ double ldcs_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ cdouble ldcs_val(const cdouble *p) {
    double2 v = __ldcs(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cfloat ldcs_val(const cfloat *p) {
    float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}

// FP32 counterpart of an FP64 element type, and the FP64 element type of
// an FP32 one (refined mode).
template <typename T> struct wide_of { using type = T; };
template <> struct wide_of<float> { using type = double; };
template <> struct wide_of<cfloat> { using type = cdouble; };
template <typename T> struct is_narrow { static constexpr bool value = false; };
template <> struct is_narrow<float> { static constexpr bool value = true; };
template <> struct is_narrow<cfloat> { static constexpr bool value = true; };

__device__ __forceinline__ float narrow_scaled(double v, double s) { return (float)(v * s); }
__device__ __forceinline__ cfloat narrow_scaled(cdouble v, double s) {
    return {(float)(v.re * s), (float)(v.im * s)};
}

// SELL-32 product over this thread's slices: for every row,
// y = sum_k a_{row,k} xin[col_k], then epi(row, y, acc).  One warp per
// 32-row slice, slices gwarp, gwarp + nwarps, ...
template <typename T, typename Epi, typename AccArr>
__device__ __forceinline__ void sell_spmv(int64_t nslices, const int64_t *slice_ptr, const int32_t *scol,
                                          const T *sval, const T *xin, int64_t gwarp, int64_t nwarps,
                                          int lane, Epi epi, AccArr &acc) {
    for (int64_t s = gwarp; s < nslices; s += nwarps) {
        const int64_t off = __ldg(slice_ptr + s);
        const int w = (int)((__ldg(slice_ptr + s + 1) - off) >> 5);
        const int32_t *cp = scol + off + lane;
        const T *vp = sval + off + lane;
        T sum{};
        int k = 0;
        for (; k + 4 <= w; k += 4) {
            int32_t cc[4];
            T vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cc[u] = __ldcs(cp + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < 4; ++u) vv[u] = ldcs_val(vp + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < 4; ++u) sum = efma(vv[u], xin[cc[u]], sum);
        }
        if (k < w) {
            int32_t cc[3];
            T vv[3];
#pragma unroll
            for (int u = 0; u < 3; ++u)
                if (k + u < w) cc[u] = __ldcs(cp + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < 3; ++u)
                if (k + u < w) vv[u] = ldcs_val(vp + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < 3; ++u)
                if (k + u < w) sum = efma(vv[u], xin[cc[u]], sum);
        }
        epi(s * 32 + lane, sum, acc);
    }
}

// Coefficient from reduced sums (re[, im]).
template <typename T>
__device__ __forceinline__ typename coef_of<T>::type mk_coef(const double *v) {
    if constexpr (is_cx<T>::value) return cdouble{v[0], v[1]};
    else return v[0];
}

// Synchronisation state of one CTA within the team of CTAs that solves one
// system: the whole grid (a single solve), or the CTA alone (a batch, one
// system per CTA).  Every CTA of a team passes the same sequence of
// barriers and reductions, so `epoch` and the slots advance in lock step.
// Several engines in one kernel share one GridSync.
struct GridSync {
    unsigned nblocks;   // CTAs in the team
    unsigned bid;       // this CTA's rank in the team
    BarrierState *bar;
    double *partials;   // [2][kMaxSums][gridDim]
    double *red;        // shared, 2 * 32 * kMaxSums
    int *sflag;         // shared
    uint64_t timeout_ns;
    unsigned epoch;
    int slot, rslot;
    bool ok;            // false once a barrier failed

    // Team = the whole grid.
    __device__ GridSync(BarrierState *b, double *p, double *r, int *f, uint64_t to)
        : nblocks(gridDim.x), bid(blockIdx.x), bar(b), partials(p), red(r), sflag(f), timeout_ns(to), epoch(0),
          slot(0), rslot(0), ok(true) {}
    // Team = this CTA alone.
    __device__ GridSync(double *r, int *f)
        : nblocks(1), bid(0), bar(nullptr), partials(nullptr), red(r), sflag(f), timeout_ns(0), epoch(0), slot(0),
          rslot(0), ok(true) {}

    // Thread 0 arrives/waits; all threads of the CTA then proceed.  Returns
    // false (uniformly) when the barrier failed.
    __device__ __forceinline__ bool gbar() {
        if (threadIdx.x == 0) *sflag = grid_arrive_wait(bar, epoch, nblocks, timeout_ns) ? 1 : 0;
        __syncthreads();
        if (*sflag == 0) { ok = false; return false; }
        return true;
    }

    // Sum K values over the grid; every thread of every CTA receives the
    // same bits.  Order: warp xor-tree, warps in index order (one CTA) or a
    // warp xor-tree over the warp totals, then over the CTAs: lane l adds
    // CTAs l, l+32, ... in order, then an xor-tree over the lanes.
    template <int K>
    __device__ __forceinline__ bool reduce(double (&v)[K]) {
        const int lane = threadIdx.x & 31;
        const int warp = threadIdx.x >> 5;
        const int nw = blockDim.x >> 5;
        warp_sum<K>(v);
        double *sr = red + rslot * (32 * kMaxSums);
        rslot ^= 1;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) sr[k * 32 + warp] = v[k];
        }
        __syncthreads();
        if (nblocks == 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double t = 0.0;
                for (int w = 0; w < nw; ++w) t += sr[k * 32 + w];
                v[k] = t;
            }
            return true;
        }
        const unsigned G = nblocks;
        double *part = partials + (size_t)slot * kMaxSums * G;
        if (warp == 0) {
            double t[K];
#pragma unroll
            for (int k = 0; k < K; ++k) t[k] = lane < nw ? sr[k * 32 + lane] : 0.0;
            warp_sum<K>(t);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) part[(size_t)k * G + bid] = t[k];
            }
        }
        if (!gbar()) return false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (unsigned b = lane; b < G; b += 32) t += part[(size_t)k * G + b];
            v[k] = t;
        }
        warp_sum<K>(v);
        slot ^= 1;
        return true;
    }

    __device__ __forceinline__ bool sync() {
        __syncthreads();
        if (nblocks == 1) return true;
        return gbar();
    }
};

template <typename T>
struct Engine {
    using S = typename coef_of<T>::type;                      // FP64 coefficient
    using ACC = typename real_of<T>::type;                    // thread accumulator
    static constexpr int DS = dslots<T>();
    static constexpr int PW = Pack<T>::W;

    const SysView<T> &sys;
    const SolveCtl &ctl;
    // CTA geometry
    int64_t gtid, gstride, gwarp, nwarps, nchunk;
    int lane;
    GridSync &gs;
    // shared memory
    S *c;            // kMaxN
    S *bt;           // kMaxN
    Acct *acct;      // accounting, kept by thread 0 (uniform in the grid)

    __device__ Engine(const SysView<T> &s, const SolveCtl &k, GridSync &g, S *c_, S *bt_, Acct *acct_)
        : sys(s), ctl(k), gs(g), c(c_), bt(bt_), acct(acct_) {
        gtid = (int64_t)g.bid * blockDim.x + threadIdx.x;
        gstride = (int64_t)g.nblocks * blockDim.x;
        gwarp = gtid >> 5;
        nwarps = gstride >> 5;
        lane = threadIdx.x & 31;
        nchunk = s.ld / PW;
    }
    __device__ __forceinline__ void op(int which, int cnt = 1) {
        if (threadIdx.x == 0) acct->ops[which] += cnt;
    }

    __device__ __forceinline__ const T *Qc(int k) const { return sys.Q + (int64_t)k * sys.ld; }
    __device__ __forceinline__ const T *Fc(int k) const { return sys.F + (int64_t)k * sys.ld; }
    __device__ __forceinline__ T *Gc(int k) const { return sys.G + (int64_t)k * sys.ld; }
    __device__ __forceinline__ T *Wc(int k) const { return sys.W + (int64_t)k * sys.ld; }

    __device__ __forceinline__ void vbytes(int nvec) {
        if (threadIdx.x == 0) acct->bytes += (double)nvec * (double)sys.N * sizeof(T);
    }
    __device__ __forceinline__ void sbytes(int nextra) {
        // SpMV: entries (value + column index), row_ptr-equivalent, x read
        // once, y written once, plus `nextra` epilogue vectors.
        if (threadIdx.x == 0) {
            acct->bytes += (double)sys.nnz * (sizeof(T) + 4) + 4.0 * (double)(sys.N + 1) +
                           (2.0 + nextra) * (double)sys.N * sizeof(T);
            acct->spmv++;
        }
    }

    template <int K>
    __device__ __forceinline__ bool reduce(double (&v)[K]) { return gs.template reduce<K>(v); }
    __device__ __forceinline__ bool sync() { return gs.sync(); }

    // Streaming pass: fn(chunk, acc) for every 16-byte chunk owned by this
    // thread, then a grid reduction of K accumulators.
    template <int K, typename Fn>
    __device__ __forceinline__ bool vsum(Fn fn, double (&out)[K]) {
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        for (int64_t ch = gtid; ch < nchunk; ch += gstride) fn(ch, acc);
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = (double)acc[k];
        return reduce<K>(out);
    }
    template <typename Fn>
    __device__ __forceinline__ bool vpass(Fn fn) {
        ACC dummy[1];
        for (int64_t ch = gtid; ch < nchunk; ch += gstride) fn(ch, dummy);
        return sync();
    }

    // SELL-32 SpMV pass over this thread's slices.
    template <int K, typename Epi>
    __device__ __forceinline__ void spmv_rows(const T *xin, Epi epi, ACC (&acc)[K]) {
        sell_spmv(sys.nslices, sys.slice_ptr, sys.scol, sys.sval, xin, gwarp, nwarps, lane, epi, acc);
    }

    // ------------------------------------------------------------------
    // passes
    // ------------------------------------------------------------------

    // r = b - A x, g_0 = r; sums ||b||^2, ||r||^2, q_1^H r.
    __device__ __noinline__ bool ph_residual(double &bb, double &rr, S &qr, bool write_g0) {
        constexpr int K = 2 + DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        const T *q1 = Qc(0);
        T *g0 = Gc(0);
        spmv_rows<K>(sys.x, [&](int64_t row, T y, ACC(&a)[K]) {
            T bv = sys.b[row];
            T rv = subT(bv, y);
            sys.r[row] = rv;
            if (write_g0) g0[row] = rv;
            acc_nrm(&a[0], bv);
            acc_nrm(&a[1], rv);
            acc_dot(&a[2], ldg_val(q1 + row), rv);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v)) return false;
        bb = v[0];
        rr = v[1];
        qr = mk_coef<T>(v + 2);
        sbytes(write_g0 ? 4 : 3);
        return true;
    }

    // Refined mode, inner start with x_0 = 0: b = r = g_0 = src * scale
    // (src is the FP64 residual of the outer iteration), x = 0; sums
    // ||b||^2, ||r||^2, q_1^H r.
    __device__ __noinline__ bool ph_init_narrow(const typename wide_of<T>::type *src, double scale, double &bb,
                                                double &rr, S &qr) {
        using TW = typename wide_of<T>::type;
        constexpr int K = 2 + DS;
        static_assert(PW * sizeof(TW) == 32, "a chunk of the FP32 vector is two 16-byte source loads");
        const T *q1 = Qc(0);
        T *g0 = Gc(0);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            const uint4 *sp = reinterpret_cast<const uint4 *>(src) + 2 * ch;
            uint4 w2[2] = {sp[0], sp[1]};
            TW tw[PW];
            memcpy(tw, w2, sizeof(tw));
            Pack<T> p, zero;
            Pack<T> qq = ldp_ro(q1, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                p.e[e] = narrow_scaled(tw[e], scale);
                zero.e[e] = T{};
            }
            stp(sys.b, ch, p);
            stp(sys.r, ch, p);
            stp(g0, ch, p);
            stp(sys.x, ch, zero);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                acc_nrm(&acc[0], p.e[e]);
                acc_nrm(&acc[1], p.e[e]);
                acc_dot(&acc[2], qq.e[e], p.e[e]);
            }
        }, v);
        if (!okk) return false;
        bb = v[0];
        rr = v[1];
        qr = mk_coef<T>(v + 2);
        if (threadIdx.x == 0) acct->bytes += (double)sys.N * (sizeof(TW) + 5.0 * sizeof(T));
        return true;
    }

    // w_slot = A g_slot; returns c = q_qcol^H w.
    __device__ __noinline__ bool ph_spmv_c(int sl, int qcol, S &cval) {
        constexpr int K = DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        const T *q = Qc(qcol);
        T *w = Wc(sl);
        spmv_rows<K>(Gc(sl), [&](int64_t row, T y, ACC(&a)[K]) {
            w[row] = y;
            acc_dot(&a[0], ldg_val(q + row), y);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v)) return false;
        cval = mk_coef<T>(v);
        sbytes(1);
        return true;
    }

    // z = A u (u held in r); sums z^H z, z^H u.
    __device__ __noinline__ bool ph_spmv_z(double &zz, S &zu) {
        constexpr int K = 1 + DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        spmv_rows<K>(sys.r, [&](int64_t row, T y, ACC(&a)[K]) {
            sys.z[row] = y;
            acc_nrm(&a[0], y);
            acc_dot(&a[1], y, sys.r[row]);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v)) return false;
        zz = v[0];
        zu = mk_coef<T>(v + 1);
        sbytes(1);
        return true;
    }

    // x += alpha g_sl, r -= alpha w_sl; sums ||r||^2, q_qcol^H r and
    // (when f0) f_1^H r.
    __device__ __noinline__ bool ph_alpha(S alpha, int sl, int qcol, bool f0, double &rr, S &qr, S &fr) {
        constexpr int K = 1 + 2 * DS;
        const T a = to_t<T>(alpha), na = to_t<T>(-alpha);
        const T *gp = Gc(sl);
        const T *wp = Wc(sl);
        const T *qp = qcol >= 0 ? Qc(qcol) : nullptr;
        const T *fp = f0 ? Fc(0) : nullptr;
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> xx = ldp(sys.x, ch), gg = ldp(gp, ch), rv = ldp(sys.r, ch), ww = ldp(wp, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                xx.e[e] = efma(a, gg.e[e], xx.e[e]);
                rv.e[e] = efma(na, ww.e[e], rv.e[e]);
            }
            stp(sys.x, ch, xx);
            stp(sys.r, ch, rv);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_nrm(&acc[0], rv.e[e]);
            if (qp) {
                Pack<T> qq = ldp_ro(qp, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[1], qq.e[e], rv.e[e]);
            }
            if (fp) {
                Pack<T> ff = ldp_ro(fp, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[1 + DS], ff.e[e], rv.e[e]);
            }
        }, v);
        if (!okk) return false;
        rr = v[0];
        qr = mk_coef<T>(v + 1);
        fr = mk_coef<T>(v + 1 + DS);
        vbytes(6 + (qp ? 1 : 0) + (fp ? 1 : 0));
        return true;
    }

    // x += omega u, r = u - omega z (u in r); sums ||r||^2, q_1^H r.
    __device__ __noinline__ bool ph_omega(S omega, double &rr, S &qr) {
        constexpr int K = 1 + DS;
        const T om = to_t<T>(omega), nom = to_t<T>(-omega);
        const T *qp = Qc(0);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> xx = ldp(sys.x, ch), uu = ldp(sys.r, ch), zz = ldp(sys.z, ch);
            Pack<T> qq = ldp_ro(qp, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                xx.e[e] = efma(om, uu.e[e], xx.e[e]);
                uu.e[e] = efma(nom, zz.e[e], uu.e[e]);
            }
            stp(sys.x, ch, xx);
            stp(sys.r, ch, uu);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                acc_nrm(&acc[0], uu.e[e]);
                acc_dot(&acc[1], qq.e[e], uu.e[e]);
            }
        }, v);
        if (!okk) return false;
        rr = v[0];
        qr = mk_coef<T>(v + 1);
        vbytes(6);
        return true;
    }

    // z_w = r + bt0 * w_sl (in place); sums q_qcol^H z_w.
    __device__ __noinline__ bool ph_w_first(S bt0, int sl, int qcol, S &d) {
        constexpr int K = DS;
        const T b0 = to_t<T>(bt0);
        T *wp = Wc(sl);
        const T *qp = Qc(qcol);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> rv = ldp(sys.r, ch), ww = ldp(wp, ch), qq = ldp_ro(qp, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) ww.e[e] = efma(b0, ww.e[e], rv.e[e]);
            stp(wp, ch, ww);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_dot(&acc[0], qq.e[e], ww.e[e]);
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(4);
        return true;
    }

    // z_w += bts * w_s (in place); sums q_qcol^H z_w.
    __device__ __noinline__ bool ph_w_round(S bts, int s, int sl, int qcol, S &d) {
        constexpr int K = DS;
        const T bb = to_t<T>(bts);
        T *wp = Wc(sl);
        const T *ws = Wc(s);
        const T *qp = Qc(qcol);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> zw = ldp(wp, ch), w2 = ldp(ws, ch), qq = ldp_ro(qp, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) zw.e[e] = efma(bb, w2.e[e], zw.e[e]);
            stp(wp, ch, zw);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_dot(&acc[0], qq.e[e], zw.e[e]);
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(4);
        return true;
    }

    // Last pass of the z_w sweep, fused with every deferred g-update of the
    // sweep and the omega-correction:
    //   first=true : z_w = r + bt[sl] w_sl                (empty s-loop)
    //   first=false: z_w += bt[last] w_last
    //   g = bt[sl] g_sl;  g += bt[t] g_t for t = sl+1..n-1;  g = z_w - g/omega
    // sums f_1^H g when with_f.
    __device__ __noinline__ bool ph_w_last(bool first, int sl, S inv_omega, bool with_f, S &d) {
        constexpr int K = DS;
        const int n = sys.n;
        const int last = n - 1;
        T *wp = Wc(sl);
        T *gp = Gc(sl);
        const T *wl = Wc(last);
        const T bl = to_t<T>(bt[first ? sl : last]);
        const T b0 = to_t<T>(bt[sl]);
        const T nio = to_t<T>(-inv_omega);
        const T *fp = with_f ? Fc(0) : nullptr;
        const int t0 = sl + 1;
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> zw = ldp(wp, ch), g = ldp(gp, ch);
            if (first) {
                Pack<T> rv = ldp(sys.r, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) zw.e[e] = efma(bl, zw.e[e], rv.e[e]);
            } else {
                Pack<T> w2 = ldp(wl, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) zw.e[e] = efma(bl, w2.e[e], zw.e[e]);
            }
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = emul(b0, g.e[e]);
            for (int t = t0; t < n; ++t) {
                const T bb = to_t<T>(bt[t]);
                Pack<T> gt = ldp(sys.G + (int64_t)t * sys.ld, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, gt.e[e], g.e[e]);
            }
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = efma(nio, g.e[e], zw.e[e]);
            stp(wp, ch, zw);
            stp(gp, ch, g);
            if (fp) {
                Pack<T> ff = ldp_ro(fp, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[0], ff.e[e], g.e[e]);
            }
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(5 + (n - t0) + (fp ? 1 : 0));
        return true;
    }

    // g_sl += beta g_s; sums f_fcol^H g_sl when fcol >= 0 (else no sum).
    __device__ __noinline__ bool ph_f_round(S beta, int s, int sl, int fcol, S &d) {
        const T bb = to_t<T>(beta);
        T *gp = Gc(sl);
        const T *gs = Gc(s);
        if (fcol < 0) {
            bool okk = vpass([&](int64_t ch, ACC *) {
                Pack<T> g = ldp(gp, ch), g2 = ldp(gs, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], g.e[e]);
                stp(gp, ch, g);
            });
            vbytes(3);
            return okk;
        }
        constexpr int K = DS;
        const T *fp = Fc(fcol);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> g = ldp(gp, ch), g2 = ldp(gs, ch), ff = ldp_ro(fp, ch);
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], g.e[e]);
            stp(gp, ch, g);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_dot(&acc[0], ff.e[e], g.e[e]);
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(4);
        return true;
    }

    // Block 0: g_sl = r + beta g_0; sums f_fcol^H g_sl when fcol >= 0.
    __device__ __noinline__ bool ph_g_j0(S beta, int sl, int fcol, S &d) {
        const T bb = to_t<T>(beta);
        T *gp = Gc(sl);
        const T *g0 = Gc(0);
        if (fcol < 0) {
            bool okk = vpass([&](int64_t ch, ACC *) {
                Pack<T> rv = ldp(sys.r, ch), g2 = ldp(g0, ch), g;
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], rv.e[e]);
                stp(gp, ch, g);
            });
            vbytes(3);
            return okk;
        }
        constexpr int K = DS;
        const T *fp = Fc(fcol);
        double v[K];
        bool okk = vsum<K>([&](int64_t ch, ACC *acc) {
            Pack<T> rv = ldp(sys.r, ch), g2 = ldp(g0, ch), ff = ldp_ro(fp, ch), g;
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], rv.e[e]);
            stp(gp, ch, g);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_dot(&acc[0], ff.e[e], g.e[e]);
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(4);
        return true;
    }

    // ------------------------------------------------------------------
    // helpers
    // ------------------------------------------------------------------

    __device__ __forceinline__ void record(bool rec, int64_t iter, double err) {
        if (rec && ctl.err_hist && iter < ctl.hist_cap && gs.bid == 0 && threadIdx.x == 0)
            ctl.err_hist[iter] = err;
    }

    // ------------------------------------------------------------------
    // one call of the method (Algorithm 7.1, M = I) from the current x
    // ------------------------------------------------------------------
    struct Out {
        int flag;
        int64_t iter;
        int j, i;
        double err;
    };

    // `init` (refined mode only): start from x_0 = 0 with b = init * scale
    // instead of reading b and x.
    __device__ Out inner(int64_t maxit, bool rec, double tol,
                         const typename wide_of<T>::type *init = nullptr, double scale = 1.0) {
        const int n = sys.n;
        Out o{1, 0, 0, 0, 0.0};
        if (threadIdx.x == 0)
            for (int q = 0; q < 5; ++q) acct->ops[q] = 0;

        // r_0 = b - A x_0 (step 2) with the stopping-rule denominator
        double bb, rr;
        S e, fr{}, d{};
        bool started = false;
        if constexpr (is_narrow<T>::value) {
            if (init) {
                if (!ph_init_narrow(init, scale, bb, rr, e)) return o;
                op(OP_NORM, 2);
                started = true;
            }
        }
        if (!started) {
            if (!ph_residual(bb, rr, e, true)) return o;
            op(OP_NORM, 2);
            op(OP_MATVEC, 1);
        }
        double bnrm2 = sqrt(bb);
        if (bnrm2 == 0.0) bnrm2 = 1.0;
        double err = sqrt(rr) / bnrm2;
        o.err = err;
        record(rec, 0, err);
        if (err < tol) { o.flag = 0; return o; }

        // w_0 = A g_0, c_0 = q_1^H w_0; e_0 = q_1^H r_0 came with r_0
        S cv;
        if (!ph_spmv_c(0, 0, cv)) return o;
        op(OP_MATVEC);
        op(OP_DOT);
        if (threadIdx.x == 0) c[0] = cv;
        __syncthreads();
        if (is_zero(cv) || !finite_of(cv)) { o.flag = -1; return o; }
        op(OP_DOT);

        S omega{}, inv_omega{};
        int64_t iter = 0;
        for (int j = 0;; ++j) {
            o.j = j;
            for (int i = 1; i <= n - 1; ++i) {
                o.i = i;
                // steps 5-8: alpha, x, r, e (and f_1^H r in block 0)
                S alpha = e / c[i - 1];
                double r2;
                S qr;
                if (!ph_alpha(alpha, i - 1, i, j == 0, r2, qr, fr)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = sqrt(r2) / bnrm2;
                o.err = err;
                iter++;
                o.iter = iter;
                record(rec, iter, err);
                if (err < tol) { o.flag = 0; return o; }
                if (iter >= maxit) return o;
                e = qr;
                op(OP_DOT);

                if (j >= 1) {
                    // steps 10-18: sweep the rest of block j-1 with q's
                    S b0 = -(e / c[i]);
                    if (threadIdx.x == 0) bt[i] = b0;
                    __syncthreads();
                    op(OP_SAXPY);
                    op(OP_SCALE);
                    if (i == n - 1) {
                        if (!ph_w_last(true, i, inv_omega, true, d)) return o;
                    } else {
                        if (!ph_w_first(b0, i, i + 1, d)) return o;
                        for (int s = i + 1; s <= n - 1; ++s) {
                            S bs = -(d / c[s]);
                            if (threadIdx.x == 0) bt[s] = bs;
                            __syncthreads();
                            op(OP_DOT);
                            op(OP_SAXPY, 2);
                            if (s < n - 1) {
                                if (!ph_w_round(bs, s, i, s + 1, d)) return o;
                            } else {
                                if (!ph_w_last(false, i, inv_omega, true, d)) return o;
                            }
                        }
                    }
                    op(OP_SAXPY);   // omega-correction
                    // steps 19-22: sweep block j with f's
                    for (int s = 0; s <= i - 1; ++s) {
                        S beta = -(d / c[s]);
                        op(OP_DOT);
                        op(OP_SAXPY);
                        if (!ph_f_round(beta, s, i, s + 1 <= i - 1 ? s + 1 : -1, d)) return o;
                    }
                } else {
                    // steps 24-29 (block 0)
                    S beta = -(fr / c[0]);
                    op(OP_DOT);
                    op(OP_SAXPY);
                    if (!ph_g_j0(beta, i, i >= 2 ? 1 : -1, d)) return o;
                    for (int s = 1; s <= i - 1; ++s) {
                        beta = -(d / c[s]);
                        op(OP_DOT);
                        op(OP_SAXPY);
                        if (!ph_f_round(beta, s, i, s + 1 <= i - 1 ? s + 1 : -1, d)) return o;
                    }
                }
                // steps 31-32: w = A g, c = q_{i+1}^H w
                if (!ph_spmv_c(i, i, cv)) return o;
                op(OP_MATVEC);
                op(OP_DOT);
                if (threadIdx.x == 0) c[i] = cv;
                __syncthreads();
                if (is_zero(cv) || !finite_of(cv)) { o.flag = -1; return o; }
            }

            // steps 34-36: alpha, x, u (u kept in r)
            o.i = n;
            {
                S alpha = e / c[n - 1];
                double u2;
                S dummy;
                if (!ph_alpha(alpha, n - 1, -1, false, u2, dummy, fr)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = sqrt(u2) / bnrm2;
                o.err = err;
                if (err < tol) {
                    iter++;
                    o.iter = iter;
                    record(rec, iter, err);
                    o.flag = 0;
                    return o;
                }
                // step 38: omega = (A u)^H u / ||A u||^2, Eq. 5.1 guard
                double zz;
                S zu;
                if (!ph_spmv_z(zz, zu)) return o;
                op(OP_MATVEC);
                op(OP_DOT);
                if (zz == 0.0 || !isfinite(zz)) { o.flag = -1; return o; }
                op(OP_DOT);
                omega = zu / zz;
                if (ctl.kappa > 0.0) {
                    op(OP_NORM, 2);
                    double arho = abs_of(zu) / (sqrt(zz) * sqrt(u2));
                    if (arho < ctl.kappa && arho != 0.0) omega = (ctl.kappa * omega) / arho;
                }
                if (is_zero(omega) || !finite_of(omega)) { o.flag = -1; return o; }
                inv_omega = recip(omega);
                // steps 39-41: x += omega u, r = u - omega A u, e = q_1^H r
                S q1r;
                double r2;
                if (!ph_omega(omega, r2, q1r)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = sqrt(r2) / bnrm2;
                o.err = err;
                iter++;
                o.iter = iter;
                record(rec, iter, err);
                if (err < tol) { o.flag = 0; return o; }
                if (iter >= maxit) return o;
                e = q1r;
                op(OP_DOT);
            }
            // steps 42-50: sweep block j with q's into slot 0
            {
                S b0 = -(e / c[0]);
                if (threadIdx.x == 0) bt[0] = b0;
                __syncthreads();
                op(OP_SAXPY);
                op(OP_SCALE);
                if (n == 1) {
                    if (!ph_w_last(true, 0, inv_omega, false, d)) return o;
                } else {
                    if (!ph_w_first(b0, 0, 1, d)) return o;
                    for (int s = 1; s <= n - 1; ++s) {
                        S bs = -(d / c[s]);
                        if (threadIdx.x == 0) bt[s] = bs;
                        __syncthreads();
                        op(OP_DOT);
                        op(OP_SAXPY, 2);
                        if (s < n - 1) {
                            if (!ph_w_round(bs, s, 0, s + 1, d)) return o;
                        } else {
                            if (!ph_w_last(false, 0, inv_omega, false, d)) return o;
                        }
                    }
                }
                op(OP_SAXPY);   // omega-correction
                // step 51: w = A g, c = q_1^H w
                if (!ph_spmv_c(0, 0, cv)) return o;
                op(OP_MATVEC);
                op(OP_DOT);
                if (threadIdx.x == 0) c[0] = cv;
                __syncthreads();
                if (is_zero(cv) || !finite_of(cv)) { o.flag = -1; return o; }
            }
        }
    }
};

}  // namespace mlb
