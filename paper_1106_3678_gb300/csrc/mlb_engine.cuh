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
// Work distribution: every CTA of the team owns a contiguous, balanced range
// of 32-row slices (and the matching rows of every vector).  Every pass
// reads its streamed operands through a TMA-fed shared-memory tile
// pipeline (one producer warp, 15 consumer warps): vector chunks for the
// streaming passes, SELL slices (values and columns) for the SpMV, whose
// consumers gather x directly.
// Every vector a CTA bulk-loads was last written by that same CTA (its own
// rows) or is read-only.
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

#include <type_traits>

#include "mlb_device.cuh"
#include "mlb_tiles.cuh"

namespace mlb {

constexpr int kThreads = kTileThreads;   // 15 consumer warps + 1 producer warp
constexpr int kMaxN = 64;       // largest number of shadow vectors
constexpr int kMaxSums = 8;     // doubles reduced per pass (max)
constexpr int kRedDoubles = kMaxSums * (kThreads / 2 + 1);   // shared reduction scratch

// Result record written by CTA 0 at the end of a solve.
struct DevResult {
    int32_t flag, j, i, status;
    int64_t iter, spmv, outer;
    double err, true_relres, bytes;
    int64_t ops[5];
    double flops;
    int32_t ctas, pad;   // CTAs that solved the system
};

enum { OP_MATVEC = 0, OP_DOT = 1, OP_SAXPY = 2, OP_SCALE = 3, OP_NORM = 4 };

// Per-CTA accounting in shared memory (identical in every CTA).
struct Acct {
    int64_t ops[5];   // Table 4.3 categories of the current inner call
    int64_t spmv;     // all sparse products of the solve
    // Algorithmic bytes and floating-point operations of the solve, kept
    // in integer arithmetic: thread 0 adds to them in every pass, on the
    // pass's critical path, where FP64 adds would cost ~60 cycles each.
    int64_t bytes;
    int64_t flops;
    // Scalars evaluated by thread 0 and read by every thread after a
    // __syncthreads: FP64 division and square root are costly on this GPU,
    // so they are not repeated by all threads.  Calls rotate through the
    // slots, so a slot is rewritten only after three more __syncthreads,
    // which every reader of its previous value has already passed.
    double d[4];
    cdouble z[4];
};

// ILU(0) preconditioner M = L U of Algorithm 7.1 (the preconditioner of
// the paper's experiments, §5), stored in A's pattern: in row i, entries
// before the diagonal are L's (unit diagonal implied), the rest U's.  The
// solve iterates on y = M x, with every product A M^{-1} v formed as
// A (M^{-1} v).  Rows are grouped by level for the triangular solves: a
// row of level l depends only on rows of lower levels (of L, or of U taken
// from the last row upwards).  lu == nullptr: no ILU(0) preconditioner.
template <typename T>
struct IluView {
    const int64_t *rp;          // N+1; columns increase within each row
    const int32_t *ci;
    const T *lu;
    const int32_t *dpos;        // position of row i's diagonal, relative to rp[i]
    const int32_t *lrows;       // rows of L's levels: level l = lrows[lptr[l] .. lptr[l+1])
    const int32_t *lptr;
    const int32_t *urows;       // rows of U's levels
    const int32_t *uptr;
    int nlev_l, nlev_u;
    int64_t nnz;
    T *t;                       // ld: M^{-1} of the current product's input
    // the same rows in level-position order: entry count and the first
    // kIluEll entries of position q at e * N + q, U's diagonal at q
    const int32_t *lcnt, *ucnt, *lell_c, *uell_c;
    const T *lell_a, *uell_a, *udiag;
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
    int spt[3];                 // slices per SpMV tile with 0, 1, 2 epilogue vectors (<= 0: no tiles)
    int ew;                     // 1: scalar entries; 3: 3x3-block entries (three values, one column)
    int narrow_rows;            // no slice is wider than 7 entries (blocks)
    const T *Q;                 // ld x n
    const T *F;                 // ld x (n-1), F = A^H Q(:,0:n-2)
    T *G, *W;                   // ld x n rings
    T *x, *r, *z;               // ld
    T *b;                       // ld (written only by the refined-mode inner start)
    int n;
    IluView<T> ilu;             // ILU(0) preconditioner (ilu.lu == nullptr: none)
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
// Loads through L2 only: values another CTA wrote since the last team
// barrier (an SM's L1 may still hold an older copy of the line).
__device__ __forceinline__ double ldcg_val(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_val(const float *p) { return __ldcg(p); }
__device__ __forceinline__ cdouble ldcg_val(const cdouble *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cfloat ldcg_val(const cfloat *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
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

// Balanced contiguous share [lo, hi) of `total` items for member `bid` of
// `nblocks`.
__device__ __forceinline__ void own_range(int64_t total, unsigned nblocks, unsigned bid, int64_t &lo, int64_t &hi) {
    lo = total * (int64_t)bid / nblocks;
    hi = total * (int64_t)(bid + 1) / nblocks;
}

// One SELL-32 slice (32 rows, width w, entries at slice offset `off`):
// the row sum of this lane, for slices of any width.
template <typename T>
__device__ __forceinline__ T sell_slice_sum(const int32_t *cp, const T *vp, int w, const T *xin) {
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
    return sum;
}

// 3x3-block storage ("triplet" SELL-32): entry k of lane l holds the three
// values of the lane's row in one 3x3 block, a_{row,c}, a_{row,c+1},
// a_{row,c+2}, at vp[3 (32 k)] .. (lane-strided by 96), and the block's first
// column c at cp[32 k]: one column index per three values.  The row sum is
// taken value by value in column order, which is the order of the row's
// scalar entries when the blocks are listed by block column.
template <typename T>
__device__ __forceinline__ T sell_slice_sum3(const int32_t *cp, const T *vp, int w, const T *xin) {
    T sum{};
    for (int k = 0; k < w; ++k) {
        const int32_t c = __ldcs(cp + 32 * k);
        const T v0 = ldcs_val(vp + 96 * k), v1 = ldcs_val(vp + 96 * k + 1), v2 = ldcs_val(vp + 96 * k + 2);
        sum = efma(v0, xin[c], sum);
        sum = efma(v1, xin[c + 1], sum);
        sum = efma(v2, xin[c + 2], sum);
    }
    return sum;
}
template <typename T>
__device__ __noinline__ T sell_slice_sum3_wide(const int32_t *cp, const T *vp, int w, const T *xin) {
    T sum{};
    for (int k = 0; k < w; ++k) {
        const int32_t c = cp[32 * k];
        const T x0 = xin[c], x1 = xin[c + 1], x2 = xin[c + 2];
        sum = efma(vp[96 * k], x0, sum);
        sum = efma(vp[96 * k + 1], x1, sum);
        sum = efma(vp[96 * k + 2], x2, sum);
    }
    return sum;
}

// Row sum of a slice wider than the pipelined path takes, from a stage
// (values at vp, column indices at cp, lane-strided by 32).  Out of line
// so that its registers do not weigh on the pipelined loop.
template <typename T>
__device__ __noinline__ T sell_slice_sum_wide(const int32_t *cp, const T *vp, int w, const T *xin) {
    T sum{};
    int k = 0;
    for (; k + 8 <= w; k += 8) {
        T xw[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xw[u] = xin[cp[32 * (k + u)]];
#pragma unroll
        for (int u = 0; u < 8; ++u) sum = efma(vp[32 * (k + u)], xw[u], sum);
    }
    if (k < w) {
        T xw[7];
#pragma unroll
        for (int u = 0; u < 7; ++u)
            if (k + u < w) xw[u] = xin[cp[32 * (k + u)]];
#pragma unroll
        for (int u = 0; u < 7; ++u)
            if (k + u < w) sum = efma(vp[32 * (k + u)], xw[u], sum);
    }
    return sum;
}

// SELL-32 product over the slices [s_lo, s_hi) owned by this CTA: for
// every row, y = sum_k a_{row,k} xin[col_k], then fin(row, y, e, acc) where
// e[i] = epi[i][row] for the NE epilogue vectors (rows of this CTA).  The
// producer warp streams tiles of `spt` slices (values, column indices and
// the epilogue entries of the tile's rows) into the shared-memory ring;
// consumer warp w takes slice w of each tile.  Each warp is
// software-pipelined across tiles: the x gathers of tile t+1 are issued
// between the FMAs of tile t (each gather reuses the register its FMA has
// just read), so the FP64 pipe and the memory system work at the same time
// and the only global loads on a warp's critical path are the gathers.
// The epilogue's stores are fenced for later bulk (async-proxy) reads.
// EW = 3: the 3x3-block storage (see sell_slice_sum3); slice offsets and
// widths then count blocks.  Slices up to PW entries wide take the
// pipelined path (PW registers of gathered x per thread), wider ones a
// direct loop.  Returns false when a tile wait timed out.
template <int NE, int EW = 1, int PW = 8, typename T, typename Fin, typename AccArr>
__device__ __forceinline__ bool sell_spmv(TileRing *R, unsigned &pseq, unsigned &cseq, uint64_t timeout_ns,
                                          int64_t s_lo, int64_t s_hi, int spt, const int64_t *slice_ptr,
                                          const int32_t *scol, const T *sval, const T *xin,
                                          const T *const (&epi)[NE > 0 ? NE : 1], int lane, Fin fin,
                                          AccArr &acc) {
    static_assert(EW == 1 || EW == 3, "scalar entries or 3x3 blocks");
    constexpr int kPipeW = PW;
    constexpr int NEA = NE > 0 ? NE : 1;
    const int cw = threadIdx.x >> 5;
    const SliceOffsets off(R, slice_ptr, s_lo, s_hi);
    bool ok = true;
    if (spt <= 0) {
        // slices too wide for one stage: direct loads, no pipeline
        if (cw < kConsumerWarps) {
            for (int64_t s = s_lo + cw; s < s_hi; s += kConsumerWarps) {
                const int64_t o = off(s);
                const int w = (int)((off(s + 1) - o) >> 5);
                const int64_t row = s * 32 + lane;
                T e[NEA];
#pragma unroll
                for (int i = 0; i < NE; ++i) e[i] = epi[i][row];
                if constexpr (EW == 3)
                    fin(row, sell_slice_sum3(scol + o + lane, sval + 3 * (o + lane), w, xin), e, acc);
                else
                    fin(row, sell_slice_sum(scol + o + lane, sval + o + lane, w, xin), e, acc);
            }
        }
        fence_proxy_async_global();
        return true;
    }
    if (cw == kConsumerWarps) {
        if (lane == 0) {
            const void *ep[NEA];
#pragma unroll
            for (int i = 0; i < NE; ++i) ep[i] = epi[i];
            ok = produce_sell(R, s_lo, s_hi, spt, off, sval, EW * (int)sizeof(T), (int)sizeof(T), scol, ep, NE, pseq,
                              timeout_ns);
        }
        return ok;
    }
    // one slice of one tile, as seen by this warp: stage, entry offset of
    // the slice in the stage (o), entries of the tile (nv), slice width w
    // (w < 0: no slice for this warp in this tile)
    struct Job {
        int st, o, nv, w;
    };
    const int nt = (int)((s_hi - s_lo + spt - 1) / spt);
    // copies in registers (the epilogue's generic stores could alias them)
    unsigned char *const rbuf = R->buf;
    const unsigned cs0 = cseq;
    auto stage_of = [&](const Job &j) { return rbuf + (size_t)j.st * kStageBytes; };
    auto vals = [&](const Job &j) { return reinterpret_cast<const T *>(stage_of(j)) + EW * (j.o + lane); };
    auto cols = [&](const Job &j) {
        return reinterpret_cast<const int32_t *>(stage_of(j) + (size_t)j.nv * EW * sizeof(T)) + j.o + lane;
    };
    // epilogue entry i of this warp's row in the tile
    auto epv = [&](const Job &j, int i) {
        return reinterpret_cast<const T *>(stage_of(j) + (size_t)j.nv * (EW * sizeof(T) + 4))[(i * spt + cw) * 32 +
                                                                                             lane];
    };
    // wait for tile t and locate this warp's slice in it
    auto locate = [&](int t, Job &j) -> bool {
        const unsigned q = cs0 + (unsigned)t;
        j.st = (int)(q % kStages);
        j.o = j.nv = 0;
        j.w = -1;
        if (!mbar_wait(&R->full[j.st], (q / kStages) & 1u, timeout_ns)) return false;
        const int64_t s0 = s_lo + (int64_t)t * spt;
        const int64_t s1 = s0 + spt < s_hi ? s0 + spt : s_hi;
        const int64_t s = s0 + cw;
        if (s < s1) {
            const int64_t e0 = off(s0), es = off(s);
            j.nv = (int)(off(s1) - e0);
            j.o = (int)(es - e0);
            j.w = (int)((off(s + 1) - es) >> 5);
        }
        return true;
    };
    auto row_of = [&](int t) { return (s_lo + (int64_t)t * spt + cw) * 32 + lane; };
    int done = 0;
    // x gathers of slice j into xv (pipelined path: widths up to kPipeW)
    auto gather = [&](const Job &j, T (&xv)[kPipeW * EW]) {
        if (j.w >= 0 && j.w <= kPipeW) {
            const int32_t *cp = cols(j);
#pragma unroll
            for (int u = 0; u < kPipeW; ++u)
                if (u < j.w) {
                    const int32_t c = cp[32 * u];
#pragma unroll
                    for (int q = 0; q < EW; ++q) xv[EW * u + q] = xin[c + q];
                }
        }
    };
    // Tile t (slice jc, its x in xc): the FMAs, each followed by the gather
    // of slice jn (tile t+1, when `more`) into the register it has just
    // read; then the epilogue and the release of the stage.  (Gathering two
    // tiles ahead measured slower: 228 against 206 us per iteration at 128^3.)
    auto step = [&](int t, const Job &jc, T (&xc)[kPipeW * EW], const Job &jn, bool more) {
        const bool na = jc.w >= 0 && jc.w <= kPipeW;
        const bool nb = more && jn.w >= 0 && jn.w <= kPipeW;
        const T *va = vals(jc);
        const int32_t *cb = cols(jn);
        T sum{};
#pragma unroll
        for (int u = 0; u < kPipeW; ++u) {
            if (na && u < jc.w) {
#pragma unroll
                for (int q = 0; q < EW; ++q) sum = efma(va[32 * EW * u + q], xc[EW * u + q], sum);
            }
            if (nb && u < jn.w) {
                const int32_t c = cb[32 * u];
#pragma unroll
                for (int q = 0; q < EW; ++q) xc[EW * u + q] = xin[c + q];
            }
        }
        if (jc.w > kPipeW) {
            if constexpr (EW == 3) sum = sell_slice_sum3_wide(cols(jc), va, jc.w, xin);
            else sum = sell_slice_sum_wide(cols(jc), va, jc.w, xin);
        }
        if (jc.w >= 0) {
            T e[NEA];
#pragma unroll
            for (int i = 0; i < NE; ++i) e[i] = epv(jc, i);
            fin(row_of(t), sum, e, acc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&R->empty[jc.st]);
        ++done;
    };
    if (nt > 0) {
        Job ja, jb;
        T xv[kPipeW * EW];
        ok = locate(0, ja);
        if (ok) gather(ja, xv);
        for (int t = 0; ok && t < nt; ++t) {
            const bool more = t + 1 < nt;
            if (more && !locate(t + 1, jb)) {
                ok = false;
                break;
            }
            step(t, ja, xv, jb, more);
            ja = jb;
        }
    }
    cseq = cs0 + (unsigned)done;
    fence_proxy_async_global();
    return ok;
}

// A 16-byte chunk of input i of a tile, from shared memory.
template <typename T>
__device__ __forceinline__ Pack<T> lds(const unsigned char *stage, int tc, int i, int k) {
    Pack<T> p;
    *reinterpret_cast<uint4 *>(&p) = *reinterpret_cast<const uint4 *>(stage + ((size_t)i * tc + k) * 16);
    return p;
}

// Coefficient from reduced sums (re[, im]).
template <typename T>
__device__ __forceinline__ typename coef_of<T>::type mk_coef(const double *v) {
    if constexpr (is_cx<T>::value) return cdouble{v[0], v[1]};
    else return v[0];
}

// Synchronisation state of one CTA within the team of CTAs that solves one
// system: the whole grid (a single solve), a group of CTAs of a batch
// launch (a large system of a batch), or the CTA alone (the other systems
// of a batch).  Every CTA of a team passes the same sequence of
// barriers and reductions, so `epoch` and the slots advance in lock step.
// Several engines in one kernel share one GridSync.
//
// The object lives in shared memory, one per CTA (thread-private copies
// would sit in local memory, which the L1 left beside the tile ring cannot
// hold for 512 threads, so every access would go to L2).  Writers: `epoch`
// and `slot` thread 0; `ok` any thread (only ever set to false).  The tile
// sequence counters are per thread, in `seqs[threadIdx.x]` (the producer
// lane counts issued tiles, a consumer thread consumed ones): one shared
// counter would race, since in a pass of at most kStages tiles a fast warp
// can finish the pass before a slow one has read where it starts.
struct GridSync {
    unsigned nblocks;   // CTAs in the team
    unsigned bid;       // this CTA's rank in the team
    BarrierState *bar;
    double *partials;   // [2][kMaxSums][gridDim]
    double *red;        // shared, kRedDoubles
    int *sflag;         // shared
    uint64_t timeout_ns;
    unsigned epoch;
    int slot;
    bool ok;            // false once a barrier or a tile wait failed
    TileRing *ring;     // shared-memory tile pipeline of this CTA
    unsigned *seqs;     // shared, kThreads per-thread tile counters

    __device__ __forceinline__ unsigned &seq() const { return seqs[threadIdx.x]; }

    // Team = the whole grid.
    __device__ GridSync(BarrierState *b, double *p, double *r, int *f, uint64_t to, TileRing *rg, unsigned *sq)
        : nblocks(gridDim.x), bid(blockIdx.x), bar(b), partials(p), red(r), sflag(f), timeout_ns(to), epoch(0),
          slot(0), ok(true), ring(rg), seqs(sq) {}
    // Team = `nb` CTAs of a batch launch (rank `id`) with their own
    // barrier state and partial sums ([2][kMaxSums][nb] doubles).
    __device__ GridSync(BarrierState *b, double *p, unsigned nb, unsigned id, double *r, int *f, uint64_t to,
                        TileRing *rg, unsigned *sq)
        : nblocks(nb), bid(id), bar(b), partials(p), red(r), sflag(f), timeout_ns(to), epoch(0), slot(0), ok(true),
          ring(rg), seqs(sq) {}
    // Team = this CTA alone.
    __device__ GridSync(double *r, int *f, uint64_t to, TileRing *rg, unsigned *sq)
        : nblocks(1), bid(0), bar(nullptr), partials(nullptr), red(r), sflag(f), timeout_ns(to), epoch(0), slot(0),
          ok(true), ring(rg), seqs(sq) {}

    // Thread 0 arrives/waits; all threads of the CTA then proceed.  Returns
    // false (uniformly) when the barrier failed.
    __device__ __forceinline__ bool gbar() {
        if (threadIdx.x == 0) *sflag = grid_arrive_wait(bar, epoch, nblocks, timeout_ns) ? 1 : 0;
        __syncthreads();
        if (*sflag == 0) { ok = false; return false; }
        return true;
    }

    // Sum K values over the team; every thread of every CTA receives the
    // same bits.  A dependent FP64 add costs about 60 cycles on this GPU and
    // one warp issues at most one FP64 instruction per ~60 cycles, so the
    // sums are short trees spread over many warps, independent sums
    // interleaved:
    //   CTA level 0: lanes l < 16 of every warp add their value to lane
    //                l+16's (256 partials per sum);
    //   CTA level 1: task (k, g), g < 64, on its own thread, adds partials
    //                g, g+64, g+128, g+192 as a pair tree;
    //   CTA level 2: warp k adds the 64 level-1 results of sum k (lane l:
    //                l and l+32), then an xor tree over the lanes;
    //   team:        with several CTAs, warp k of every CTA adds the CTA
    //                totals of sum k the same way (lane l: CTAs l, l+32, ...
    //                as a pair tree, then the xor tree).
    // Fixed order for a given team size: deterministic.
    template <int K>
    __device__ __forceinline__ bool reduce(double (&v)[K]) {
        static_assert(K <= kMaxSums && kThreads == 512, "reduction layout");
        constexpr int P0 = kThreads / 2, G1 = P0 / 4;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        double *sv = red;                     // K * P0 partials
        double *bc = red + kMaxSums * P0;     // K totals
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double h = v[k] + __shfl_down_sync(0xffffffffu, v[k], 16);
            if (lane < 16) sv[k * P0 + warp * 16 + lane] = h;
        }
        __syncthreads();
        for (int task = tid; task < K * G1; task += kThreads) {
            double *p = sv + (task / G1) * P0 + task % G1;
            const double a0 = p[0], a1 = p[G1], a2 = p[2 * G1], a3 = p[3 * G1];
            p[0] = (a0 + a1) + (a2 + a3);      // only this task reads slot 0
        }
        __syncthreads();
        if (warp < K) {
            const double *p = sv + warp * P0 + lane;
            double t = p[0] + p[32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) bc[warp] = t;
        }
        __syncthreads();
        if (nblocks == 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = bc[k];
            return true;
        }
        const unsigned G = nblocks;
        double *part = partials + (size_t)slot * kMaxSums * G;
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) part[(size_t)k * G + bid] = bc[k];
        }
        if (!gbar()) return false;
        if (tid == 0) slot ^= 1;   // every thread has read it (gbar synchronises)
        if (warp < K) {
            const double *p = part + (size_t)warp * G;
            double t = 0.0;
            for (unsigned b0 = 0; b0 < G; b0 += 256) {
                double x[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const unsigned b = b0 + lane + 32 * m;
                    x[m] = b < G ? p[b] : 0.0;
                }
                const double s8 = ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
                t = b0 == 0 ? s8 : t + s8;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) bc[warp] = t;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = bc[k];
        return true;
    }

    __device__ __forceinline__ bool sync() {
        __syncthreads();
        if (nblocks == 1) return true;
        return gbar();
    }

    // sync() in two halves: arrive() once this CTA's writes are done,
    // wait() before reading other CTAs' writes; work between the two that
    // reads nothing written in this step overlaps the wait.  Every thread
    // calls both; wait() returns false (uniformly) when the barrier failed.
    __device__ __forceinline__ void arrive() {
        __syncthreads();
        if (nblocks > 1 && threadIdx.x == 0) grid_arrive(bar, epoch);
    }
    __device__ __forceinline__ bool wait() {
        if (nblocks == 1) return true;   // arrive()'s __syncthreads ordered the CTA
        if (threadIdx.x == 0) *sflag = grid_wait(bar, epoch, nblocks, timeout_ns) ? 1 : 0;
        __syncthreads();
        if (*sflag == 0) { ok = false; return false; }
        return true;
    }
};

// A call of Engine::inner without residual replacement (every solve but
// the refined mode's FP32 inner one).
struct NoHook {
    static constexpr bool kActive = false;
};

// PC: built with the ILU(0) preconditioner passes (ilu_pre and the
// product passes' switch to M^{-1} of their input); without it none of
// that code is reachable.  EW: the matrix storage of the products (1:
// scalar SELL-32; 3: 3x3 blocks, see sell_slice_sum3).
template <typename T, bool PC = false, int EW = 1>
struct Engine {
    using S = typename coef_of<T>::type;                      // FP64 coefficient
    using ACC = typename real_of<T>::type;                    // thread accumulator
    static constexpr int DS = dslots<T>();
    static constexpr int PW = Pack<T>::W;
    static constexpr int CPS = 32 * sizeof(T) / 16;           // 16-byte chunks per slice

    const SysView<T> &sys;
    const SolveCtl &ctl;
    GridSync &gs;
    // shared memory
    S *c;            // kMaxN
    S *bt;           // kMaxN
    Acct *acct;      // accounting, kept by thread 0 (uniform in the grid)
    // ownership: slices [s_lo, s_hi), chunks [c_lo, c_hi)
    int64_t s_lo, s_hi, c_lo, c_hi;

    // Constructed by one thread in shared memory (one engine per CTA; see
    // GridSync); every thread then calls attach().
    __device__ Engine(const SysView<T> &s, const SolveCtl &k, GridSync &g, S *c_, S *bt_, Acct *acct_)
        : sys(s), ctl(k), gs(g), c(c_), bt(bt_), acct(acct_) {
        own_range(s.nslices, g.nblocks, g.bid, s_lo, s_hi);
        c_lo = s_lo * CPS;
        c_hi = s_hi * CPS;
    }
    __device__ void attach() { soff_load(gs.ring, sys.slice_ptr, s_lo, s_hi); }
    // Counts one Table 4.3 operation and its algorithmic floating-point
    // operations (real arithmetic): a product 2 per stored entry; an inner
    // product, AXPY or norm 2 per element; a scaling 1 per element.
    // Complex values: a multiply-add is 8 real operations, |v|^2 4, a
    // scaling 6.
    __device__ __forceinline__ void op(int which, int cnt = 1) {
        if (threadIdx.x == 0) {
            acct->ops[which] += cnt;
            constexpr bool cx_ = is_cx<T>::value;
            const int64_t N = sys.N;
            int64_t f;
            if (which == OP_MATVEC) f = (cx_ ? 8 : 2) * sys.nnz;
            else if (which == OP_SCALE) f = (cx_ ? 6 : 1) * N;
            else if (which == OP_NORM) f = (cx_ ? 4 : 2) * N;
            else f = (cx_ ? 8 : 2) * N;
            acct->flops += cnt * f;
        }
    }

    // Evaluate fn() in thread 0 only and give the value to every thread.
    // Back-to-back calls use rotating slots; `bs` is the caller's counter
    // (a register, the same sequence in every thread).
    template <typename Fn>
    __device__ __forceinline__ S once_s(unsigned &bs, Fn fn) {
        const int k = bs++ & 3;
        if constexpr (is_cx<T>::value) {
            if (threadIdx.x == 0) acct->z[k] = fn();
            __syncthreads();
            return acct->z[k];
        } else {
            if (threadIdx.x == 0) acct->d[k] = fn();
            __syncthreads();
            return acct->d[k];
        }
    }
    template <typename Fn>
    __device__ __forceinline__ double once_d(unsigned &bs, Fn fn) {
        const int k = bs++ & 3;
        if (threadIdx.x == 0) acct->d[k] = fn();
        __syncthreads();
        return acct->d[k];
    }

    __device__ __forceinline__ const T *Qc(int k) const { return sys.Q + (int64_t)k * sys.ld; }
    __device__ __forceinline__ const T *Fc(int k) const { return sys.F + (int64_t)k * sys.ld; }
    __device__ __forceinline__ T *Gc(int k) const { return sys.G + (int64_t)k * sys.ld; }
    __device__ __forceinline__ T *Wc(int k) const { return sys.W + (int64_t)k * sys.ld; }

    __device__ __forceinline__ void vbytes(int nvec) {
        if (threadIdx.x == 0) acct->bytes += nvec * sys.N * (int64_t)sizeof(T);
    }
    __device__ __forceinline__ void sbytes(int nextra) {
        // SpMV: entries (values, and a column index per stored entry of EW
        // values), row_ptr-equivalent, x read once, y written once, plus
        // `nextra` epilogue vectors.
        if (threadIdx.x == 0) {
            acct->bytes += sys.nnz * (int64_t)sizeof(T) + sys.nnz / EW * 4 + 4 * (sys.N + 1) +
                           (2 + nextra) * sys.N * (int64_t)sizeof(T);
            acct->spmv++;
        }
    }

    template <int K>
    __device__ __forceinline__ bool reduce(double (&v)[K]) { return gs.template reduce<K>(v); }
    __device__ __forceinline__ bool sync() { return gs.sync(); }

    // Inputs of a streaming pass: only the producer lane reads the list (it
    // issues the copies); every thread derives the tile geometry from the
    // count, so the consumers keep it in registers.
    struct PassIn {
        const T *const *in;
        int ni;
    };
    __device__ __forceinline__ TileGeom geom(const PassIn &P) const {
        return TileGeom{tile_chunks_for(P.ni), c_lo, c_hi};
    }
    // The producer lane's copy descriptor.
    __device__ __forceinline__ void tile_pass(TilePass &D, const PassIn &P) const {
        D.ni = P.ni;
        for (int i = 0; i < P.ni; ++i) D.in[i] = P.in[i];
        D.tc = tile_chunks_for(P.ni);
        D.c_lo = c_lo;
        D.c_hi = c_hi;
    }

    // Streaming pass through the tile pipeline: fn(chunk, stage, k, acc)
    // for every chunk of this CTA, then a team reduction of K sums.
    template <int K, typename Fn>
    __device__ __forceinline__ bool tsum(const PassIn &P, Fn fn, double (&out)[K]) {
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        bool okw = true;
        TileRing *const ring = gs.ring;
        const uint64_t to = gs.timeout_ns;
        if ((threadIdx.x >> 5) == kConsumerWarps) {
            if ((threadIdx.x & 31) == 0) {
                TilePass D;
                tile_pass(D, P);
                unsigned sq = gs.seq();
                okw = produce(ring, D, sq, to);
                gs.seq() = sq;
            }
        } else {
            unsigned sq = gs.seq();
            okw = consume(ring, geom(P), sq, to, [&](int64_t ch, const unsigned char *st, int k) { fn(ch, st, k, acc); });
            gs.seq() = sq;
        }
        if (!okw) gs.ring->failed = 1;
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = (double)acc[k];
        if (!reduce<K>(out)) return false;
        if (gs.ring->failed) { gs.ok = false; return false; }
        return true;
    }
    // Streaming pass with no inner product: the tiles, then only a team
    // barrier (the next pass gathers what this one wrote), no reduction.
    template <typename Fn>
    __device__ __forceinline__ bool tpass(const PassIn &P, Fn fn) {
        bool okw = true;
        TileRing *const ring = gs.ring;
        const uint64_t to = gs.timeout_ns;
        if ((threadIdx.x >> 5) == kConsumerWarps) {
            if ((threadIdx.x & 31) == 0) {
                TilePass D;
                tile_pass(D, P);
                unsigned sq = gs.seq();
                okw = produce(ring, D, sq, to);
                gs.seq() = sq;
            }
        } else {
            unsigned sq = gs.seq();
            okw = consume(ring, geom(P), sq, to, [&](int64_t ch, const unsigned char *st, int k) { fn(ch, st, k); });
            gs.seq() = sq;
        }
        if (!okw) gs.ring->failed = 1;
        if (!sync()) return false;
        if (gs.ring->failed) { gs.ok = false; return false; }
        return true;
    }

    // SELL-32 SpMV pass over the owned slices (matrix tiles through the
    // ring).  A failed tile wait marks the ring; the pass's reduction then
    // reports it.
    template <int K, int NE, typename Fin>
    __device__ __forceinline__ void spmv_rows(const T *xin, const T *const (&epi)[NE], Fin fin, ACC (&acc)[K]) {
        // with ILU(0) the product is A t, t = M^{-1} xin formed by the
        // caller (ilu_pre) before the pass
        if constexpr (PC) {
            if (sys.ilu.lu) xin = sys.ilu.t;
        }
        unsigned sq = gs.seq();   // issued (producer lane) or consumed (consumers) tiles
        bool okw;
        // FP32 and complex engines: a pipelined width of 7 where the rows
        // allow it (gathered x registers fewer: the refined solve 3 %, the
        // complex one 3.5 % less time per iteration); the real FP64 engine
        // keeps 8 (no gain at 7)
        if constexpr (is_narrow<T>::value || is_cx<T>::value) {
            if (sys.narrow_rows)
                okw = sell_spmv<NE, EW, 7>(gs.ring, sq, sq, gs.timeout_ns, s_lo, s_hi, sys.spt[NE], sys.slice_ptr,
                                           sys.scol, sys.sval, xin, epi, threadIdx.x & 31, fin, acc);
            else
                okw = sell_spmv<NE, EW>(gs.ring, sq, sq, gs.timeout_ns, s_lo, s_hi, sys.spt[NE], sys.slice_ptr,
                                        sys.scol, sys.sval, xin, epi, threadIdx.x & 31, fin, acc);
        } else {
            okw = sell_spmv<NE, EW>(gs.ring, sq, sq, gs.timeout_ns, s_lo, s_hi, sys.spt[NE], sys.slice_ptr,
                                    sys.scol, sys.sval, xin, epi, threadIdx.x & 31, fin, acc);
        }
        gs.seq() = sq;
        if (!okw) gs.ring->failed = 1;
    }
    __device__ __forceinline__ bool ring_ok() {
        if (gs.ring->failed) { gs.ok = false; return false; }
        return true;
    }

    // ------------------------------------------------------------------
    // ILU(0) preconditioner (Algorithm 7.1 with M = L U)
    // ------------------------------------------------------------------

    // One row of a triangular solve, loaded ahead: its index, up to
    // kIluReg entries (column, factor value) in registers, where the rest
    // of its entries start and end, and the row's right-hand-side entry
    // (forward) or its U diagonal (backward).  i < 0: no row.
    static constexpr int kIluReg = 4;   // == kIluEll (entries stored by position)
    struct IluRow {
        int i, cnt;
        int64_t rest, end;
        int32_t c[kIluReg];
        T a[kIluReg];
        T v;
    };
    // Row q of L's level order (forward: entries before the diagonal).
    // Its count and first entries are read by position, independently of
    // the row index; entries beyond kIluReg come from the pattern.
    __device__ __forceinline__ void ilu_fetch_l(int64_t q, int64_t hi, const T *v, IluRow &R) const {
        R.i = -1;
        if (q >= hi) return;
        const IluView<T> &M = sys.ilu;
        const int64_t N = sys.N;
        const int i = M.lrows[q];
        const int n = M.lcnt[q];
        const int cnt = n < kIluReg ? n : kIluReg;
#pragma unroll
        for (int e = 0; e < kIluReg; ++e)
            if (e < cnt) {
                R.c[e] = M.lell_c[e * N + q];
                R.a[e] = M.lell_a[e * N + q];
            }
        R.i = i;
        R.cnt = cnt;
        R.rest = R.end = 0;
        if (n > kIluReg) {
            R.rest = M.rp[i] + kIluReg;
            R.end = M.rp[i] + n;
        }
        R.v = v[i];
    }
    // Row q of U's level order (backward: entries after the diagonal).
    __device__ __forceinline__ void ilu_fetch_u(int64_t q, int64_t hi, IluRow &R) const {
        R.i = -1;
        if (q >= hi) return;
        const IluView<T> &M = sys.ilu;
        const int64_t N = sys.N;
        const int i = M.urows[q];
        const int n = M.ucnt[q];
        const int cnt = n < kIluReg ? n : kIluReg;
#pragma unroll
        for (int e = 0; e < kIluReg; ++e)
            if (e < cnt) {
                R.c[e] = M.uell_c[e * N + q];
                R.a[e] = M.uell_a[e * N + q];
            }
        R.i = i;
        R.cnt = cnt;
        R.rest = R.end = 0;
        if (n > kIluReg) {
            const int64_t d = M.rp[i] + M.dpos[i];
            R.rest = d + 1 + kIluReg;
            R.end = d + 1 + n;
        }
        R.v = M.udiag[q];
    }
    // s - sum of a_e out[c_e] over the row's entries, in pattern order.
    __device__ __forceinline__ T ilu_row_sum(const IluRow &R, T s, const T *out) const {
        const IluView<T> &M = sys.ilu;
#pragma unroll
        for (int e = 0; e < kIluReg; ++e)
            if (e < R.cnt) s = efma(-R.a[e], ldcg_val(out + R.c[e]), s);
        for (int64_t k = R.rest; k < R.end; ++k) s = efma(-M.lu[k], ldcg_val(out + M.ci[k]), s);
        return s;
    }

    // out = M^{-1} v: L z = v by forward substitution (unit diagonal), then
    // U out = z by backward substitution, in place.  Level scheduling: all
    // rows of one level at once over the team's threads, a team barrier
    // between levels.  Each row is one sequential sum in pattern order, as
    // in the definition; U's diagonal divides.  A thread's first row of the
    // next level (index, entries, right-hand side or diagonal) does not
    // depend on the current level, so it is loaded while the barrier is
    // pending, and only the values of earlier levels are read after it.
    __device__ __noinline__ bool ilu_solve(const T *v, T *out) {
        const IluView<T> &M = sys.ilu;
        // a level's positions split into one contiguous chunk per CTA of
        // ceil(size / CTAs): every CTA shares each level (a level is a few
        // thousand scattered rows), and a warp reads consecutive positions
        const int64_t G = gs.nblocks, bid = gs.bid;
        const int tid = threadIdx.x;
        auto chunk = [&](const int32_t *ptr, int l, int64_t &q0, int64_t &q1) {
            const int64_t lo = ptr[l], hi = ptr[l + 1], ch = (hi - lo + G - 1) / G;
            q0 = lo + bid * ch;
            q1 = q0 + ch < hi ? q0 + ch : hi;
        };
        const int nl = M.nlev_l, nu = M.nlev_u;
        int64_t q0, q1;
        IluRow R;
        chunk(M.lptr, 0, q0, q1);
        ilu_fetch_l(q0 + tid, q1, v, R);
        for (int l = 0; l < nl; ++l) {
            if (R.i >= 0) out[R.i] = ilu_row_sum(R, R.v, out);
            for (int64_t q = q0 + tid + kThreads; q < q1; q += kThreads) {   // more rows than threads
                const int i = M.lrows[q];
                const int64_t k0 = M.rp[i], kd = k0 + M.dpos[i];
                T t = v[i];
                for (int64_t k = k0; k < kd; ++k) t = efma(-M.lu[k], ldcg_val(out + M.ci[k]), t);
                out[i] = t;
            }
            gs.arrive();
            if (l + 1 < nl) {
                chunk(M.lptr, l + 1, q0, q1);
                ilu_fetch_l(q0 + tid, q1, v, R);
            } else {
                chunk(M.uptr, 0, q0, q1);
                ilu_fetch_u(q0 + tid, q1, R);
            }
            if (!gs.wait()) return false;
        }
        for (int l = 0; l < nu; ++l) {
            if (R.i >= 0) out[R.i] = ilu_row_sum(R, ldcg_val(out + R.i), out) / R.v;
            for (int64_t q = q0 + tid + kThreads; q < q1; q += kThreads) {
                const int i = M.urows[q];
                const int64_t kd = M.rp[i] + M.dpos[i], k1 = M.rp[i + 1];
                T t = ldcg_val(out + i);
                for (int64_t k = kd + 1; k < k1; ++k) t = efma(-M.lu[k], ldcg_val(out + M.ci[k]), t);
                out[i] = t / M.lu[kd];
            }
            gs.arrive();
            if (l + 1 < nu) {
                chunk(M.uptr, l + 1, q0, q1);
                ilu_fetch_u(q0 + tid, q1, R);
            }
            if (!gs.wait()) return false;
        }
        if (threadIdx.x == 0) {   // factors and row data once, v read, out written and re-read
            acct->bytes += M.nnz * (int64_t)(sizeof(T) + 4) + sys.N * (int64_t)(8 + 4 + 8 + 3 * sizeof(T));
            acct->flops += (is_cx<T>::value ? 8 : 2) * M.nnz;
        }
        return true;
    }

    // Before a product pass with ILU(0): t = M^{-1} in, where `in` is the
    // pass's input vector (the pass then multiplies t).  A separate call,
    // so the product passes themselves carry no call to the solve.
    __device__ __forceinline__ bool ilu_pre(const T *in) {
        if constexpr (!PC) {
            return true;
        } else {
            if (!sys.ilu.lu) return true;
            return ilu_solve(in, sys.ilu.t);
        }
    }

    // y_0 = M x_0 = L (U x_0), in place on x: t = U x, then x = L t (two
    // row-parallel products).
    __device__ __noinline__ bool ilu_to_y() {
        const IluView<T> &M = sys.ilu;
        const int64_t nth = (int64_t)gs.nblocks * kThreads;
        const int64_t me = (int64_t)gs.bid * kThreads + threadIdx.x;
        T *const x = sys.x, *const t = M.t;
        for (int64_t i = me; i < sys.N; i += nth) {
            const int64_t kd = M.rp[i] + M.dpos[i], k1 = M.rp[i + 1];
            T s{};
            for (int64_t k = kd; k < k1; ++k) s = efma(M.lu[k], x[M.ci[k]], s);
            t[i] = s;
        }
        if (!gs.sync()) return false;
        for (int64_t i = me; i < sys.N; i += nth) {
            const int64_t k0 = M.rp[i], kd = k0 + M.dpos[i];
            T s = ldcg_val(t + i);
            for (int64_t k = k0; k < kd; ++k) s = efma(M.lu[k], ldcg_val(t + M.ci[k]), s);
            x[i] = s;
        }
        return gs.sync();
    }

    // x = M^{-1} y once the final residual pass has formed t = M^{-1} y.
    __device__ __noinline__ bool ilu_to_x() {
        const int64_t nth = (int64_t)gs.nblocks * kThreads;
        const int64_t me = (int64_t)gs.bid * kThreads + threadIdx.x;
        T *const x = sys.x;
        const T *t = sys.ilu.t;
        for (int64_t i = me; i < sys.N; i += nth) x[i] = ldcg_val(t + i);
        return gs.sync();
    }

    // ------------------------------------------------------------------
    // passes
    // ------------------------------------------------------------------

    // r = b - A x, g_0 = r; sums ||b||^2, ||r||^2, q_1^H r.
    __device__ __forceinline__ bool ph_residual_body(double &bb, double &rr, S &qr, bool write_g0) {
        constexpr int K = 2 + DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        const T *q1 = Qc(0);
        T *g0 = Gc(0);
        const T *epi[2] = {sys.b, q1};
        T *const r = sys.r;
        // epilogues capture by value: a captured reference would keep the
        // pointer in memory, reloaded after every store of the loop
        spmv_rows<K>(sys.x, epi, [=](int64_t row, T y, const T (&e)[2], ACC(&a)[K]) {
            T rv = subT(e[0], y);
            r[row] = rv;
            if (write_g0) g0[row] = rv;
            acc_nrm(&a[0], e[0]);
            acc_nrm(&a[1], rv);
            acc_dot(&a[2], e[1], rv);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v) || !ring_ok()) return false;
        bb = v[0];
        rr = v[1];
        qr = mk_coef<T>(v + 2);
        sbytes(write_g0 ? 4 : 3);
        return true;
    }

    // Refined mode, inner start with x_0 = 0: b = r = g_0 = src * scale
    // (src is the FP64 residual of the outer iteration, rows of this CTA),
    // x = 0; sums ||b||^2, ||r||^2, q_1^H r.  Direct loads (one pass per
    // outer step).
    __device__ __noinline__ bool ph_init_narrow(const typename wide_of<T>::type *src, double scale, double &bb,
                                                double &rr, S &qr) {
        using TW = typename wide_of<T>::type;
        constexpr int K = 2 + DS;
        static_assert(PW * sizeof(TW) == 32, "a chunk of the FP32 vector is two 16-byte source loads");
        const T *q1 = Qc(0);
        T *g0 = Gc(0);
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        T *const bq = sys.b;
        T *const rq = sys.r;
        T *const xq = sys.x;
        const int64_t clo = c_lo, chi = c_hi;
        if ((threadIdx.x >> 5) < kConsumerWarps) {
            for (int64_t ch = clo + threadIdx.x; ch < chi; ch += kConsumers) {
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
                stp(bq, ch, p);
                stp(rq, ch, p);
                stp(g0, ch, p);
                stp(xq, ch, zero);
#pragma unroll
                for (int e = 0; e < PW; ++e) {
                    acc_nrm(&acc[0], p.e[e]);
                    acc_nrm(&acc[1], p.e[e]);
                    acc_dot(&acc[2], qq.e[e], p.e[e]);
                }
            }
        }
        fence_proxy_async_global();
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v)) return false;
        bb = v[0];
        rr = v[1];
        qr = mk_coef<T>(v + 2);
        if (threadIdx.x == 0) acct->bytes += sys.N * (int64_t)(sizeof(TW) + 5 * sizeof(T));
        return true;
    }

    // Refined mode, residual replacement: r = src * scale, with src the
    // FP64 true residual b - A x of the outer iteration (rows of this CTA);
    // sums ||r||^2, q_qcol^H r (qcol >= 0) and, when f0, f_1^H r: the
    // inner products the step that follows the replaced update needs.
    // Direct loads.
    __device__ __noinline__ bool ph_replace_narrow(const typename wide_of<T>::type *src, double scale, int qcol,
                                                   bool f0, double &rr, S &qr, S &fr) {
        using TW = typename wide_of<T>::type;
        constexpr int K = 1 + 2 * DS;
        static_assert(PW * sizeof(TW) == 32, "a chunk of the FP32 vector is two 16-byte source loads");
        const T *qv = qcol >= 0 ? Qc(qcol) : nullptr;
        const T *fv = f0 ? Fc(0) : nullptr;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        T *const rq = sys.r;
        const int64_t clo = c_lo, chi = c_hi;
        if ((threadIdx.x >> 5) < kConsumerWarps) {
            for (int64_t ch = clo + threadIdx.x; ch < chi; ch += kConsumers) {
                const uint4 *sp = reinterpret_cast<const uint4 *>(src) + 2 * ch;
                uint4 w2[2] = {sp[0], sp[1]};
                TW tw[PW];
                memcpy(tw, w2, sizeof(tw));
                Pack<T> p;
#pragma unroll
                for (int e = 0; e < PW; ++e) p.e[e] = narrow_scaled(tw[e], scale);
                stp(rq, ch, p);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_nrm(&acc[0], p.e[e]);
                if (qv) {
                    Pack<T> qq = ldp_ro(qv, ch);
#pragma unroll
                    for (int e = 0; e < PW; ++e) acc_dot(&acc[1], qq.e[e], p.e[e]);
                }
                if (fv) {
                    Pack<T> ff = ldp_ro(fv, ch);
#pragma unroll
                    for (int e = 0; e < PW; ++e) acc_dot(&acc[1 + DS], ff.e[e], p.e[e]);
                }
            }
        }
        fence_proxy_async_global();
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v)) return false;
        rr = v[0];
        qr = mk_coef<T>(v + 1);
        fr = mk_coef<T>(v + 1 + DS);
        if (threadIdx.x == 0)
            acct->bytes += sys.N * (int64_t)(sizeof(TW) + (1 + (qv ? 1 : 0) + (fv ? 1 : 0)) * sizeof(T));
        return true;
    }

    // w_slot = A g_slot; returns c = q_qcol^H w.
    __device__ __forceinline__ bool ph_spmv_c_body(int sl, int qcol, S &cval) {
        constexpr int K = DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        const T *q = Qc(qcol);
        T *w = Wc(sl);
        const T *epi[1] = {q};
        spmv_rows<K>(Gc(sl), epi, [=](int64_t row, T y, const T (&e)[1], ACC(&a)[K]) {
            w[row] = y;
            acc_dot(&a[0], e[0], y);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v) || !ring_ok()) return false;
        cval = mk_coef<T>(v);
        sbytes(1);
        return true;
    }

    // z = A u (u held in r); sums z^H z, z^H u.
    __device__ __forceinline__ bool ph_spmv_z_body(double &zz, S &zu) {
        constexpr int K = 1 + DS;
        ACC acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = ACC(0);
        const T *epi[1] = {sys.r};
        T *const z = sys.z;
        spmv_rows<K>(sys.r, epi, [=](int64_t row, T y, const T (&e)[1], ACC(&a)[K]) {
            z[row] = y;
            acc_nrm(&a[0], y);
            acc_dot(&a[1], y, e[0]);
        }, acc);
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
        if (!reduce<K>(v) || !ring_ok()) return false;
        zz = v[0];
        zu = mk_coef<T>(v + 1);
        sbytes(1);
        return true;
    }

    // x += alpha g_sl, r -= alpha w_sl; sums ||r||^2, q_qcol^H r and
    // (when f0) f_1^H r.
    __device__ __forceinline__ bool ph_alpha_body(S alpha, int sl, int qcol, bool f0, double &rr, S &qr, S &fr) {
        constexpr int K = 1 + 2 * DS;
        const T a = to_t<T>(alpha), na = to_t<T>(-alpha);
        const bool hq = qcol >= 0;
        const T *in[6] = {sys.x, Gc(sl), sys.r, Wc(sl), hq ? Qc(qcol) : nullptr, f0 ? Fc(0) : nullptr};
        int ni = 4;
        if (hq) in[ni++] = Qc(qcol);
        if (f0) in[ni++] = Fc(0);
        const int iq = 4, iff = hq ? 5 : 4;
        T *const xo = sys.x;
        T *const ro = sys.r;
        const PassIn P{in, ni};
        const int tc = tile_chunks_for(P.ni);
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> xx = lds<T>(st, tc, 0, k), gg = lds<T>(st, tc, 1, k), rv = lds<T>(st, tc, 2, k),
                    ww = lds<T>(st, tc, 3, k);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                xx.e[e] = efma(a, gg.e[e], xx.e[e]);
                rv.e[e] = efma(na, ww.e[e], rv.e[e]);
            }
            stp(xo, ch, xx);
            stp(ro, ch, rv);
#pragma unroll
            for (int e = 0; e < PW; ++e) acc_nrm(&acc[0], rv.e[e]);
            if (hq) {
                Pack<T> qq = lds<T>(st, tc, iq, k);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[1], qq.e[e], rv.e[e]);
            }
            if (f0) {
                Pack<T> ff = lds<T>(st, tc, iff, k);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[1 + DS], ff.e[e], rv.e[e]);
            }
        }, v);
        if (!okk) return false;
        rr = v[0];
        qr = mk_coef<T>(v + 1);
        fr = mk_coef<T>(v + 1 + DS);
        vbytes(6 + (hq ? 1 : 0) + (f0 ? 1 : 0));
        return true;
    }

    // x += omega u, r = u - omega z (u in r); sums ||r||^2, q_1^H r.
    __device__ __forceinline__ bool ph_omega_body(S omega, double &rr, S &qr) {
        constexpr int K = 1 + DS;
        const T om = to_t<T>(omega), nom = to_t<T>(-omega);
        const T *in[4] = {sys.x, sys.r, sys.z, Qc(0)};
        T *const xo = sys.x;
        T *const ro = sys.r;
        const PassIn P{in, 4};
        const int tc = tile_chunks_for(P.ni);
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> xx = lds<T>(st, tc, 0, k), uu = lds<T>(st, tc, 1, k), zz = lds<T>(st, tc, 2, k),
                    qq = lds<T>(st, tc, 3, k);
#pragma unroll
            for (int e = 0; e < PW; ++e) {
                xx.e[e] = efma(om, uu.e[e], xx.e[e]);
                uu.e[e] = efma(nom, zz.e[e], uu.e[e]);
            }
            stp(xo, ch, xx);
            stp(ro, ch, uu);
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
    __device__ __forceinline__ bool ph_w_first_body(S bt0, int sl, int qcol, S &d) {
        constexpr int K = DS;
        const T b0 = to_t<T>(bt0);
        T *wp = Wc(sl);
        const T *in[3] = {sys.r, wp, Qc(qcol)};
        const PassIn P{in, 3};
        const int tc = tile_chunks_for(P.ni);
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> rv = lds<T>(st, tc, 0, k), ww = lds<T>(st, tc, 1, k), qq = lds<T>(st, tc, 2, k);
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
    __device__ __forceinline__ bool ph_w_round_body(S bts, int s, int sl, int qcol, S &d) {
        constexpr int K = DS;
        const T bb = to_t<T>(bts);
        T *wp = Wc(sl);
        const T *in[3] = {wp, Wc(s), Qc(qcol)};
        const PassIn P{in, 3};
        const int tc = tile_chunks_for(P.ni);
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> zw = lds<T>(st, tc, 0, k), w2 = lds<T>(st, tc, 1, k), qq = lds<T>(st, tc, 2, k);
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
    // sums f_1^H g when with_f.  The first kMaxInputs-4 columns g_t come
    // through the tile pipeline, any further ones by direct loads.
    __device__ __forceinline__ bool ph_w_last_body(bool first, int sl, S inv_omega, bool with_f, S &d) {
        constexpr int K = DS;
        const int n = sys.n;
        const int last = n - 1;
        T *wp = Wc(sl);
        T *gp = Gc(sl);
        const T bl = to_t<T>(bt[first ? sl : last]);
        const T b0 = to_t<T>(bt[sl]);
        const T nio = to_t<T>(-inv_omega);
        const int t0 = sl + 1;
        const int nt = n - t0;                                     // g_t columns
        const int ntile = nt < kMaxInputs - 4 ? nt : kMaxInputs - 4;
        const T *in[kMaxInputs];
        int ni = 0;
        in[ni++] = wp;
        in[ni++] = gp;
        in[ni++] = first ? sys.r : Wc(last);
        const int i_f = ni;
        if (with_f) in[ni++] = Fc(0);
        const int i_t = ni;
        for (int t = 0; t < ntile; ++t) in[ni++] = Gc(t0 + t);
        const T *const Gb = sys.G;
        const int64_t ldv = sys.ld;
        const S *const btl = bt;
        const PassIn P{in, ni};
        const int tc = tile_chunks_for(P.ni);
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> zw = lds<T>(st, tc, 0, k), g = lds<T>(st, tc, 1, k), o = lds<T>(st, tc, 2, k);
            if (first) {
#pragma unroll
                for (int e = 0; e < PW; ++e) zw.e[e] = efma(bl, zw.e[e], o.e[e]);
            } else {
#pragma unroll
                for (int e = 0; e < PW; ++e) zw.e[e] = efma(bl, o.e[e], zw.e[e]);
            }
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = emul(b0, g.e[e]);
            for (int t = 0; t < nt; ++t) {
                const T bb = to_t<T>(btl[t0 + t]);
                Pack<T> gt = t < ntile ? lds<T>(st, tc, i_t + t, k) : ldp(Gb + (int64_t)(t0 + t) * ldv, ch);
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, gt.e[e], g.e[e]);
            }
#pragma unroll
            for (int e = 0; e < PW; ++e) g.e[e] = efma(nio, g.e[e], zw.e[e]);
            stp(wp, ch, zw);
            stp(gp, ch, g);
            if (with_f) {
                Pack<T> ff = lds<T>(st, tc, i_f, k);
#pragma unroll
                for (int e = 0; e < PW; ++e) acc_dot(&acc[0], ff.e[e], g.e[e]);
            }
        }, v);
        if (!okk) return false;
        d = mk_coef<T>(v);
        vbytes(5 + nt + (with_f ? 1 : 0));
        return true;
    }

    // g_sl += beta g_s; sums f_fcol^H g_sl when fcol >= 0 (else no sum).
    __device__ __forceinline__ bool ph_f_round_body(S beta, int s, int sl, int fcol, S &d) {
        const T bb = to_t<T>(beta);
        T *gp = Gc(sl);
        const T *in[3] = {gp, Gc(s), fcol >= 0 ? Fc(fcol) : nullptr};
        const PassIn P{in, fcol >= 0 ? 3 : 2};
        const int tc = tile_chunks_for(P.ni);
        if (fcol < 0) {
            bool okk = tpass(P, [&](int64_t ch, const unsigned char *st, int k) {
                Pack<T> g = lds<T>(st, tc, 0, k), g2 = lds<T>(st, tc, 1, k);
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], g.e[e]);
                stp(gp, ch, g);
            });
            vbytes(3);
            return okk;
        }
        constexpr int K = DS;
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> g = lds<T>(st, tc, 0, k), g2 = lds<T>(st, tc, 1, k), ff = lds<T>(st, tc, 2, k);
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
    __device__ __forceinline__ bool ph_g_j0_body(S beta, int sl, int fcol, S &d) {
        const T bb = to_t<T>(beta);
        T *gp = Gc(sl);
        const T *in[3] = {sys.r, Gc(0), fcol >= 0 ? Fc(fcol) : nullptr};
        const PassIn P{in, fcol >= 0 ? 3 : 2};
        const int tc = tile_chunks_for(P.ni);
        if (fcol < 0) {
            bool okk = tpass(P, [&](int64_t ch, const unsigned char *st, int k) {
                Pack<T> rv = lds<T>(st, tc, 0, k), g2 = lds<T>(st, tc, 1, k), g;
#pragma unroll
                for (int e = 0; e < PW; ++e) g.e[e] = efma(bb, g2.e[e], rv.e[e]);
                stp(gp, ch, g);
            });
            vbytes(3);
            return okk;
        }
        constexpr int K = DS;
        double v[K];
        bool okk = tsum<K>(P, [&](int64_t ch, const unsigned char *st, int k, ACC *acc) {
            Pack<T> rv = lds<T>(st, tc, 0, k), g2 = lds<T>(st, tc, 1, k), ff = lds<T>(st, tc, 2, k), g;
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

    // The streaming passes are inlined into the FP64 engines: no saves and
    // restores of registers around the calls, whose stack sits in L2
    // beside the tile ring.  The SELL product passes stay out of line in
    // the real engines (inlined, their register demand spreads over the
    // whole loop: n = 1 took 223 instead of 193 us per iteration at 128^3,
    // and the natural-order ILU(0) solve 4 % longer) but are inlined in the
    // complex one without ILU(0) (1 % faster).  The FP32 engines call every
    // pass out of line (their kernels then compile in a fraction of the
    // time; inlining gained 2 % only where the refined mode does not
    // converge without a preconditioner).
    static constexpr bool kInlinePasses = std::is_same<T, double>::value || std::is_same<T, cdouble>::value;
    static constexpr bool kInlineProducts = std::is_same<T, cdouble>::value && !PC;
#define MLB_PASS(name, inl, params, args)                                   \
    __device__ __noinline__ bool name##_ool params { return name##_body args; } \
    __device__ __forceinline__ bool name params {                            \
        if constexpr (inl) return name##_body args;                          \
        else return name##_ool args;                                         \
    }
    MLB_PASS(ph_residual, kInlineProducts, (double &bb, double &rr, S &qr, bool write_g0), (bb, rr, qr, write_g0))
    MLB_PASS(ph_spmv_c, kInlineProducts, (int sl, int qcol, S &cval), (sl, qcol, cval))
    MLB_PASS(ph_spmv_z, kInlineProducts, (double &zz, S &zu), (zz, zu))
    MLB_PASS(ph_alpha, kInlinePasses, (S alpha, int sl, int qcol, bool f0, double &rr, S &qr, S &fr), (alpha, sl, qcol, f0, rr, qr, fr))
    MLB_PASS(ph_omega, kInlinePasses, (S omega, double &rr, S &qr), (omega, rr, qr))
    MLB_PASS(ph_w_first, kInlinePasses, (S bt0, int sl, int qcol, S &d), (bt0, sl, qcol, d))
    MLB_PASS(ph_w_round, kInlinePasses, (S bts, int s, int sl, int qcol, S &d), (bts, s, sl, qcol, d))
    MLB_PASS(ph_w_last, kInlinePasses, (bool first, int sl, S inv_omega, bool with_f, S &d), (first, sl, inv_omega, with_f, d))
    MLB_PASS(ph_f_round, kInlinePasses, (S beta, int s, int sl, int fcol, S &d), (beta, s, sl, fcol, d))
    MLB_PASS(ph_g_j0, kInlinePasses, (S beta, int sl, int fcol, S &d), (beta, sl, fcol, d))
#undef MLB_PASS

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
    // instead of reading b and x.  `hook` (refined mode only): residual
    // replacement by the FP64 outer iteration.  hook->replace(qcol, f0, rr,
    // qr, fr, conv) moves the FP32 iterate into the FP64 solution, replaces
    // r by the scaled FP64 true residual and returns ||r||^2 and the inner
    // products of the replaced r that the next step needs, and whether the
    // true residual met the outer tolerance.  It is called when the
    // recursive residual meets `tol` (instead of stopping: the inner call
    // stops only once the true residual has met the outer tolerance) and,
    // at block ends, when hook->want(err) (reliable updates); a block end
    // also ends the call when hook->stalled(iter, err).
    template <typename Hook = NoHook>
    __device__ Out inner(int64_t maxit, bool rec, double tol,
                         const typename wide_of<T>::type *init = nullptr, double scale = 1.0,
                         Hook *hook = nullptr) {
        const int n = sys.n;
        Out o{1, 0, 0, 0, 0.0};
        unsigned bsl = 0;   // rotating broadcast slot of once_s / once_d
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
            if (!ilu_pre(sys.x) || !ph_residual(bb, rr, e, true)) return o;
            op(OP_NORM, 2);
            op(OP_MATVEC, 1);
        }
        const double bnrm2 = once_d(bsl, [&] {
            double t = sqrt(bb);
            return t == 0.0 ? 1.0 : t;
        });
        double err = once_d(bsl, [&] { return sqrt(rr) / bnrm2; });
        o.err = err;
        record(rec, 0, err);
        if (err < tol) { o.flag = 0; return o; }
        if constexpr (Hook::kActive) hook->reset(err);

        // w_0 = A g_0, c_0 = q_1^H w_0; e_0 = q_1^H r_0 came with r_0
        S cv;
        if (!ilu_pre(Gc(0)) || !ph_spmv_c(0, 0, cv)) return o;
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
                S alpha = once_s(bsl, [&] { return e / c[i - 1]; });
                double r2;
                S qr;
                if (!ph_alpha(alpha, i - 1, i, j == 0, r2, qr, fr)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = once_d(bsl, [&] { return sqrt(r2) / bnrm2; });
                iter++;
                o.iter = iter;
                if constexpr (Hook::kActive) {
                    hook->track(err);
                    if (err < tol) {
                        bool conv;
                        if (!hook->replace(i, j == 0, r2, qr, fr, conv)) return o;
                        err = once_d(bsl, [&] { return sqrt(r2) / bnrm2; });
                        hook->reset(err);
                        if (conv) { o.err = err; o.flag = 0; return o; }
                    }
                }
                o.err = err;
                record(rec, iter, err);
                if (!Hook::kActive && err < tol) { o.flag = 0; return o; }
                if (iter >= maxit) return o;
                e = qr;
                op(OP_DOT);

                if (j >= 1) {
                    // steps 10-18: sweep the rest of block j-1 with q's
                    S b0 = once_s(bsl, [&] { return -(e / c[i]); });
                    if (threadIdx.x == 0) bt[i] = b0;
                    __syncthreads();
                    op(OP_SAXPY);
                    op(OP_SCALE);
                    if (i == n - 1) {
                        if (!ph_w_last(true, i, inv_omega, true, d)) return o;
                    } else {
                        if (!ph_w_first(b0, i, i + 1, d)) return o;
                        for (int s = i + 1; s <= n - 1; ++s) {
                            S bs = once_s(bsl, [&] { return -(d / c[s]); });
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
                        S beta = once_s(bsl, [&] { return -(d / c[s]); });
                        op(OP_DOT);
                        op(OP_SAXPY);
                        if (!ph_f_round(beta, s, i, s + 1 <= i - 1 ? s + 1 : -1, d)) return o;
                    }
                } else {
                    // steps 24-29 (block 0)
                    S beta = once_s(bsl, [&] { return -(fr / c[0]); });
                    op(OP_DOT);
                    op(OP_SAXPY);
                    if (!ph_g_j0(beta, i, i >= 2 ? 1 : -1, d)) return o;
                    for (int s = 1; s <= i - 1; ++s) {
                        beta = once_s(bsl, [&] { return -(d / c[s]); });
                        op(OP_DOT);
                        op(OP_SAXPY);
                        if (!ph_f_round(beta, s, i, s + 1 <= i - 1 ? s + 1 : -1, d)) return o;
                    }
                }
                // steps 31-32: w = A g, c = q_{i+1}^H w
                if (!ilu_pre(Gc(i)) || !ph_spmv_c(i, i, cv)) return o;
                op(OP_MATVEC);
                op(OP_DOT);
                if (threadIdx.x == 0) c[i] = cv;
                __syncthreads();
                if (is_zero(cv) || !finite_of(cv)) { o.flag = -1; return o; }
            }

            // steps 34-36: alpha, x, u (u kept in r)
            o.i = n;
            {
                S alpha = once_s(bsl, [&] { return e / c[n - 1]; });
                double u2;
                S dummy;
                if (!ph_alpha(alpha, n - 1, -1, false, u2, dummy, fr)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = once_d(bsl, [&] { return sqrt(u2) / bnrm2; });
                if constexpr (Hook::kActive) {
                    hook->track(err);
                    if (err < tol) {
                        // u (kept in r) replaced by the true residual; the
                        // omega step then works on the replaced u
                        bool conv;
                        S dq, df;
                        if (!hook->replace(-1, false, u2, dq, df, conv)) return o;
                        err = once_d(bsl, [&] { return sqrt(u2) / bnrm2; });
                        hook->reset(err);
                        if (conv) {
                            iter++;
                            o.iter = iter;
                            o.err = err;
                            o.flag = 0;
                            return o;
                        }
                    }
                }
                o.err = err;
                if (!Hook::kActive && err < tol) {
                    iter++;
                    o.iter = iter;
                    record(rec, iter, err);
                    o.flag = 0;
                    return o;
                }
                // step 38: omega = (A u)^H u / ||A u||^2, Eq. 5.1 guard
                double zz;
                S zu;
                if (!ilu_pre(sys.r) || !ph_spmv_z(zz, zu)) return o;
                op(OP_MATVEC);
                op(OP_DOT);
                if (zz == 0.0 || !isfinite(zz)) { o.flag = -1; return o; }
                op(OP_DOT);
                if (ctl.kappa > 0.0) op(OP_NORM, 2);
                omega = once_s(bsl, [&] {
                    S om = zu / zz;
                    if (ctl.kappa > 0.0) {
                        double arho = abs_of(zu) / (sqrt(zz) * sqrt(u2));
                        if (arho < ctl.kappa && arho != 0.0) om = (ctl.kappa * om) / arho;
                    }
                    return om;
                });
                if (is_zero(omega) || !finite_of(omega)) { o.flag = -1; return o; }
                inv_omega = once_s(bsl, [&] { return recip(omega); });
                // steps 39-41: x += omega u, r = u - omega A u, e = q_1^H r
                S q1r;
                double r2;
                if (!ph_omega(omega, r2, q1r)) return o;
                op(OP_SAXPY, 2);
                op(OP_NORM);
                err = once_d(bsl, [&] { return sqrt(r2) / bnrm2; });
                iter++;
                o.iter = iter;
                if constexpr (Hook::kActive) {
                    hook->track(err);
                    if (err < tol || hook->want(err)) {
                        bool conv;
                        S df;
                        if (!hook->replace(0, false, r2, q1r, df, conv)) return o;
                        err = once_d(bsl, [&] { return sqrt(r2) / bnrm2; });
                        hook->reset(err);
                        if (conv) { o.err = err; o.flag = 0; return o; }
                    }
                    if (hook->stalled(iter, err)) { o.err = err; return o; }
                }
                o.err = err;
                record(rec, iter, err);
                if (!Hook::kActive && err < tol) { o.flag = 0; return o; }
                if (iter >= maxit) return o;
                e = q1r;
                op(OP_DOT);
            }
            // steps 42-50: sweep block j with q's into slot 0
            {
                S b0 = once_s(bsl, [&] { return -(e / c[0]); });
                if (threadIdx.x == 0) bt[0] = b0;
                __syncthreads();
                op(OP_SAXPY);
                op(OP_SCALE);
                if (n == 1) {
                    if (!ph_w_last(true, 0, inv_omega, false, d)) return o;
                } else {
                    if (!ph_w_first(b0, 0, 1, d)) return o;
                    for (int s = 1; s <= n - 1; ++s) {
                        S bs = once_s(bsl, [&] { return -(d / c[s]); });
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
                if (!ilu_pre(Gc(0)) || !ph_spmv_c(0, 0, cv)) return o;
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
