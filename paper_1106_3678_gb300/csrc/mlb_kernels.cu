// Kernels of the ML(n)BiCGStab library (sm_103a).
#include <algorithm>
#include <new>

#include "mlb_internal.h"
#include "mlb_refine.cuh"
#include "mlb_solve.cuh"

namespace mlb {

// Solve and batch launches: the kernels with the ILU(0) passes only for
// handles that have that preconditioner.
template <typename T>
cudaError_t launch_solve(const SysView<T> &sys, const SolveCtl &ctl, int grid, cudaStream_t st) {
    if constexpr (!is_cx<T>::value) {
        if (sys.ew == 3)
            return sys.ilu.lu ? launch_solve_pc<T, true, 3>(sys, ctl, grid, st)
                              : launch_solve_pc<T, false, 3>(sys, ctl, grid, st);
    }
    return sys.ilu.lu ? launch_solve_pc<T, true>(sys, ctl, grid, st) : launch_solve_pc<T, false>(sys, ctl, grid, st);
}
template <typename T>
int solve_blocks_per_sm() {
    int a = solve_blocks_per_sm_pc<T, false>(), b = solve_blocks_per_sm_pc<T, true>();
    if constexpr (!is_cx<T>::value) {
        a = std::min(a, solve_blocks_per_sm_pc<T, false, 3>());
        b = std::min(b, solve_blocks_per_sm_pc<T, true, 3>());
    }
    return a < b ? a : b;
}
template <typename T>
cudaError_t launch_batch(const BatchItem<T> *items, const BatchPlan &plan, int grid, bool ilu, cudaStream_t st) {
    return ilu ? launch_batch_pc<T, true>(items, plan, grid, st) : launch_batch_pc<T, false>(items, plan, grid, st);
}
template <typename T>
int batch_blocks_per_sm() {
    const int a = batch_blocks_per_sm_pc<T, false>(), b = batch_blocks_per_sm_pc<T, true>();
    return a < b ? a : b;
}

// FP32-inner / FP64-refined launches: the kernels with the ILU(0) passes
// only when a system has that preconditioner.
template <typename T32, typename T64>
cudaError_t launch_refine(const SysView<T32> &sys, const RefView<T64> &rv, const SolveCtl &ctl,
                          const RefCtl &rc, int grid, cudaStream_t st) {
    if constexpr (!is_cx<T32>::value) {
        if (sys.ew == 3)
            return sys.ilu.lu ? launch_refine_pc<T32, T64, true, 3>(sys, rv, ctl, rc, grid, st)
                              : launch_refine_pc<T32, T64, false, 3>(sys, rv, ctl, rc, grid, st);
    }
    return sys.ilu.lu ? launch_refine_pc<T32, T64, true>(sys, rv, ctl, rc, grid, st)
                      : launch_refine_pc<T32, T64, false>(sys, rv, ctl, rc, grid, st);
}
template <typename T32, typename T64>
int refine_blocks_per_sm() {
    int a = refine_blocks_per_sm_pc<T32, T64, false>(), b = refine_blocks_per_sm_pc<T32, T64, true>();
    if constexpr (!is_cx<T32>::value) {
        a = std::min(a, refine_blocks_per_sm_pc<T32, T64, false, 3>());
        b = std::min(b, refine_blocks_per_sm_pc<T32, T64, true, 3>());
    }
    return a < b ? a : b;
}
template <typename T32, typename T64>
cudaError_t launch_batch_refine(const BatchItemR<T32, T64> *items, const BatchPlan &plan, int grid, bool ilu,
                                cudaStream_t st) {
    return ilu ? launch_batch_refine_pc<T32, T64, true>(items, plan, grid, st)
               : launch_batch_refine_pc<T32, T64, false>(items, plan, grid, st);
}
template <typename T32, typename T64>
int batch_refine_blocks_per_sm() {
    const int a = batch_refine_blocks_per_sm_pc<T32, T64, false>(),
              b = batch_refine_blocks_per_sm_pc<T32, T64, true>();
    return a < b ? a : b;
}

// FP64 -> FP32 copies (matrix values, Q, F); interleaved complex data is a
// sequence of doubles, so one kernel covers both.
__global__ void narrow_kernel(const double *src, float *dst, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

cudaError_t launch_narrow(const double *src, float *dst, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    narrow_kernel<<<(int)blocks, 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

// ===========================================================================
// shadow vectors: SplitMix64 at a counter, Box-Muller (cosine branch)
// ===========================================================================
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t t) {
    uint64_t z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_open0(uint64_t v) {
    return ((double)(v >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ double normal_at(uint64_t seed, uint64_t t) {
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = unit_open0(splitmix64_at(seed, 2ull * t));
    double u2 = unit_open0(splitmix64_at(seed, 2ull * t + 1ull));
    double rad = sqrt(-2.0 * log(u1));
    double ang = two_pi * u2;
    return rad * cos(ang);
}

// Entry e = col * N + orow of the original order (orow = perm[row] for a
// multicolour-ordered handle, else row) lands at (row, col).
__global__ void qgen_kernel(double *Q, int is_complex, int64_t N, int64_t ld, int n, uint64_t seed,
                            const int32_t *perm) {
    const int64_t total = N * (int64_t)n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t % N, col = t / N;
        const int64_t e = col * N + (perm ? (int64_t)perm[row] : row);
        if (is_complex) {
            double *q = Q + 2 * (col * ld + row);
            q[0] = normal_at(seed, 2ull * e);
            q[1] = normal_at(seed, 2ull * e + 1ull);
        } else {
            Q[col * ld + row] = normal_at(seed, (uint64_t)e);
        }
    }
}

cudaError_t launch_qgen(void *Q, int is_complex, int64_t N, int64_t ld, int n, uint64_t seed,
                        cudaStream_t st, const int32_t *perm) {
    int64_t total = N * (int64_t)n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    if (blocks < 1) blocks = 1;
    qgen_kernel<<<blocks, 256, 0, st>>>((double *)Q, is_complex, N, ld, n, seed, perm);
    return cudaGetLastError();
}

// Row permutation of a vector (16-byte or 8-byte values as double pairs
// or doubles): gather dst[r] = src[perm[r]] or scatter dst[perm[r]] = src[r].
template <typename V>
__global__ void permute_kernel(const V *src, V *dst, const int32_t *perm, int64_t N, int to_perm) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
        if (to_perm) dst[r] = src[perm[r]];
        else dst[perm[r]] = src[r];
    }
}

cudaError_t launch_permute(const void *src, void *dst, const int32_t *perm, int64_t N, int es, bool to_perm,
                           cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
    if (es == 16)
        permute_kernel<double2><<<grid, 256, 0, st>>>((const double2 *)src, (double2 *)dst, perm, N, to_perm ? 1 : 0);
    else
        permute_kernel<double><<<grid, 256, 0, st>>>((const double *)src, (double *)dst, perm, N, to_perm ? 1 : 0);
    return cudaGetLastError();
}

// ===========================================================================
// F = A^H Q(:, 0:m-1) from the CSR of A^H (values already conjugated)
// ===========================================================================
template <typename T>
__global__ void ahq_kernel(const int64_t *rp, const int32_t *ci, const T *av, int64_t N, int64_t ld,
                           const T *Q, T *F, int m) {
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < N;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = rp[row], k1 = rp[row + 1];
        for (int s = 0; s < m; ++s) {
            const T *q = Q + (int64_t)s * ld;
            T acc{};
            for (int64_t k = k0; k < k1; ++k) acc = efma(av[k], q[ci[k]], acc);
            F[(int64_t)s * ld + row] = acc;
        }
    }
}

template <typename T>
cudaError_t launch_ahq(const int64_t *rp, const int32_t *ci, const T *av, int64_t N, int64_t ld,
                       const T *Q, T *F, int m, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (N + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    ahq_kernel<T><<<(int)blocks, 256, 0, st>>>(rp, ci, av, N, ld, Q, F, m);
    return cudaGetLastError();
}

// ===========================================================================
// fused y = A x, d = Q^H y (all n shadow inner products)
// ===========================================================================
// Tiled form (the library's entry point): one CTA per SM, each owning a
// contiguous slice range.  The first NE columns of Q ride through the
// engine's TMA-fed SELL product as epilogue vectors, so their inner
// products are taken as each row of y is formed (FP64 arithmetic is scarce
// on this GPU: the dot products then share the product's pass instead of
// following it).  Columns beyond NE take further tile passes over the
// CTA's rows of y (written by the first pass) and up to G columns of Q at
// a time.  Every pass touches only the CTA's rows, so no grid barrier is
// needed.  Per-CTA sums go to `partials` in fixed order.
//
// A timed-out wait makes the CTA stop at the next pass boundary (decided
// CTA-wide with __syncthreads_or, so every thread takes the same barriers)
// and set its `status` slot.

// CTA sums of the first nv (<= NV) accumulators of every thread into
// out[0, nv): one shuffle level, then per value a 4-way pair tree over the
// 64 groups of 4 and a warp's xor tree (fixed order).  `scratch` holds
// NV * kThreads / 2 doubles.
template <int NV, typename ACC>
__device__ __forceinline__ void cta_sums(const ACC (&acc)[NV], int nv, double *scratch, double *out) {
    constexpr int P0 = kThreads / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // unrolled over the fixed bound so every index into acc is a constant
    // (a run-time index would put acc in local memory for the whole pass)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv) {
            const double h = (double)acc[v] + __shfl_down_sync(0xffffffffu, (double)acc[v], 16);
            if (lane < 16) scratch[v * P0 + warp * 16 + lane] = h;
        }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < nv * 64; task += kThreads) {
        double *q = scratch + (task / 64) * P0 + task % 64;
        q[0] = (q[0] + q[64]) + (q[128] + q[192]);
    }
    __syncthreads();
    for (int v = warp; v < nv; v += kThreads / 32) {
        const double *q = scratch + v * P0 + lane;
        double t = q[0] + q[32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) out[v] = t;
    }
    __syncthreads();   // scratch (the stages) is reused by the next pass
}

template <typename T, int NE, int PW>
__global__ void __launch_bounds__(kThreads, 1)
    spmv_qdot_tiled_kernel(SysView<T> sys, int spt, const T *x, T *y, T *yout, double *partials, int *status,
                           unsigned *ticket, double *d) {
    constexpr int DS = dslots<T>();
    constexpr int CPS = 32 * sizeof(T) / 16;
    // Q columns per later pass: as many accumulators as fit in registers
    // beside the tile loads (each extra pass re-reads only y)
    constexpr int G = DS == 1 ? 8 : 4;
    using ACC = typename real_of<T>::type;
    extern __shared__ unsigned char dsm[];
    __shared__ TileRing ring;
    // Programmatic dependent launch: the next product on the stream may be
    // scheduled as soon as every CTA of this one runs.  Its producer warp
    // streams only constant data (A and Q) into its own shared memory, so
    // it starts at once; every other thread waits for this grid to
    // complete before touching x, y, d or the shared partial sums, ticket
    // and status words (and the producer lane's later accesses follow the
    // consumers' through the CTA barriers).  The next product's set-up and
    // first tiles so overlap this one's tail.
    asm volatile("griddepcontrol.launch_dependents;");
    ring_init(&ring, ring_buffer(dsm));
    int64_t s_lo, s_hi;
    own_range(sys.nslices, gridDim.x, blockIdx.x, s_lo, s_hi);
    soff_load(&ring, sys.slice_ptr, s_lo, s_hi);   // constant data
    if ((threadIdx.x >> 5) != kConsumerWarps) asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint64_t to = 2000000000ull;
    const int n = sys.n;
    double *const scratch = reinterpret_cast<double *>(ring.buf);   // the stages, free between passes
    double *const part = partials + (size_t)blockIdx.x * kQdMaxN * DS;
    unsigned sq = 0;   // this thread's tile counter (issued or consumed)
    bool ok, bad;
    {
        ACC acc[NE * DS];
#pragma unroll
        for (int k = 0; k < NE * DS; ++k) acc[k] = ACC(0);
        const T *epi[NE];
#pragma unroll
        for (int m = 0; m < NE; ++m) epi[m] = sys.Q + (int64_t)m * sys.ld;
        const int64_t nrows = sys.N;
        const bool keep = n > NE;   // later passes read y back
        ok = sell_spmv<NE, 1, PW>(&ring, sq, sq, to, s_lo, s_hi, spt, sys.slice_ptr, sys.scol, sys.sval, x, epi,
                           threadIdx.x & 31,
                           [=](int64_t row, T v, const T (&e)[NE], ACC (&a)[NE * DS]) {
                               if (keep) y[row] = v;                // padded copy
                               if (row < nrows) yout[row] = v;      // the caller's y
#pragma unroll
                               for (int m = 0; m < NE; ++m) acc_dot(&a[m * DS], e[m], v);
                           },
                           acc);
        bad = __syncthreads_or(!ok);   // also: this CTA's rows of y are written and fenced
        if (!bad) cta_sums(acc, NE * DS, scratch, part);
    }
    const int64_t c_lo = s_lo * CPS, c_hi = s_hi * CPS;
    for (int g0 = NE; g0 < n && !bad; g0 += G) {
        const int ng = n - g0 < G ? n - g0 : G;
        TilePass P;
        P.ni = 1 + ng;
        P.in[0] = y;
        for (int m = 0; m < ng; ++m) P.in[1 + m] = sys.Q + (int64_t)(g0 + m) * sys.ld;
        P.tc = tile_chunks_for(P.ni);
        P.c_lo = c_lo;
        P.c_hi = c_hi;
        ACC acc[G * DS];
#pragma unroll
        for (int k = 0; k < G * DS; ++k) acc[k] = ACC(0);
        const int tc = P.tc;
        if ((threadIdx.x >> 5) == kConsumerWarps) {
            if ((threadIdx.x & 31) == 0) ok = produce(&ring, P, sq, to);
        } else {
            ok = consume(&ring, TileGeom{tc, c_lo, c_hi}, sq, to, [&](int64_t, const unsigned char *st, int k) {
                const Pack<T> yy = lds<T>(st, tc, 0, k);
#pragma unroll
                for (int m = 0; m < G; ++m) {
                    if (m < ng) {
                        const Pack<T> qq = lds<T>(st, tc, 1 + m, k);
#pragma unroll
                        for (int e = 0; e < Pack<T>::W; ++e) acc_dot(&acc[m * DS], qq.e[e], yy.e[e]);
                    }
                }
            });
        }
        bad = __syncthreads_or(!ok);   // every tile consumed: the stages are free
        if (!bad) cta_sums(acc, ng * DS, scratch, part + (size_t)g0 * DS);
    }
    if (threadIdx.x == 0) status[blockIdx.x] = bad ? 1 : 0;
    ring_drain(&ring, sq, sq, to);
    // The last CTA to finish sums every CTA's partials (fixed order, the
    // same whichever CTA it is) and ORs the status slots into d[n * DS];
    // it resets the ticket for the next launch.  No CTA waits for another.
    __shared__ int s_last;
    __threadfence();   // this CTA's partials and status before its ticket
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // one warp per value: lanes stride over the CTAs in index order, then
    // the warp's xor tree
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int v = warp; v < n * DS; v += kThreads / 32) {
            double t = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(&partials[(size_t)b * kQdMaxN * DS + v]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) d[v] = t;
        }
    }
    int st = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) st |= __ldcg(&status[b]);
    st = __syncthreads_or(st);
    if (threadIdx.x == 0) {
        d[n * DS] = st ? 1.0 : 0.0;
        *ticket = 0u;
    }
}

template <typename T, int NE, int PW>
static cudaError_t launch_qd_tiled_pw(const SysView<T> &sys, int spt, const T *x, T *y, T *yout,
                                      double *partials, int grid, int *status, unsigned *ticket, double *d,
                                      cudaEvent_t ev, cudaStream_t st) {
    cudaError_t e = allow_ring((const void *)spmv_qdot_tiled_kernel<T, NE, PW>);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev, st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kRingBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, spmv_qdot_tiled_kernel<T, NE, PW>, sys, spt, x, y, yout, partials, status,
                              ticket, d);
}

// The pipelined width of the product: 7 when no slice is wider (two
// registers of gathered x fewer than 8: 61 against 65 us per FP64 product
// at 128^3, n = 4, 7-point stencil), else 8.
template <typename T, int NE>
static cudaError_t launch_qd_tiled_ne(const SysView<T> &sys, int64_t maxw, int spt, const T *x, T *y, T *yout,
                                      double *partials, int grid, int *status, unsigned *ticket, double *d,
                                      cudaEvent_t ev, cudaStream_t st) {
    if (maxw <= 7)
        return launch_qd_tiled_pw<T, NE, 7>(sys, spt, x, y, yout, partials, grid, status, ticket, d, ev, st);
    return launch_qd_tiled_pw<T, NE, 8>(sys, spt, x, y, yout, partials, grid, status, ticket, d, ev, st);
}

template <typename T>
cudaError_t launch_spmv_qdot_tiled(const SysView<T> &sys, int ne, int64_t maxw, int spt, const T *x, T *y,
                                   T *yout, double *partials, int grid, int *status, unsigned *ticket, double *d,
                                   cudaEvent_t ev, cudaStream_t st) {
    constexpr int DS = dslots<T>();
    if (ne < 1 || ne > sys.n || (ne != 1 && ne != 2 && ne != 4) || (DS == 2 && ne > 2))
        return cudaErrorInvalidValue;
    if constexpr (DS == 1) {
        if (ne == 4)
            return launch_qd_tiled_ne<T, 4>(sys, maxw, spt, x, y, yout, partials, grid, status, ticket, d, ev, st);
    }
    if (ne == 2)
        return launch_qd_tiled_ne<T, 2>(sys, maxw, spt, x, y, yout, partials, grid, status, ticket, d, ev, st);
    return launch_qd_tiled_ne<T, 1>(sys, maxw, spt, x, y, yout, partials, grid, status, ticket, d, ev, st);
}

// ===========================================================================
// failure-detection self-test: a barrier one participant never reaches
// ===========================================================================
__global__ void barrier_selftest_kernel(BarrierState *bs, uint64_t timeout_ns) {
    __shared__ int flag;
    unsigned epoch = 0;
    grid_barrier(bs, epoch, gridDim.x + 1, timeout_ns, &flag);
}

cudaError_t launch_barrier_selftest(int grid, BarrierState *bs, uint64_t timeout_ns, cudaStream_t st) {
    void *args[] = {(void *)&bs, (void *)&timeout_ns};
    return cudaLaunchCooperativeKernel((const void *)barrier_selftest_kernel, dim3(grid), dim3(64), args, 0,
                                       st);
}

// ===========================================================================
// explicit instantiations
// ===========================================================================
// Elementwise map of a diagonal preconditioner (see launch_diag_apply).
template <typename T>
__global__ void diag_apply_kernel(T *x, const T *d, int64_t n, int divide) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = divide ? x[i] / d[i] : x[i] * d[i];
}

template <typename T>
cudaError_t launch_diag_apply(T *x, const T *d, int64_t n, bool divide, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)std::min<int64_t>(want, 152 * 16);
    diag_apply_kernel<T><<<grid, 256, 0, st>>>(x, d, n, divide ? 1 : 0);
    return cudaGetLastError();
}

template cudaError_t launch_solve<double>(const SysView<double> &, const SolveCtl &, int, cudaStream_t);
template cudaError_t launch_solve<cdouble>(const SysView<cdouble> &, const SolveCtl &, int, cudaStream_t);
template int solve_blocks_per_sm<double>();
template int solve_blocks_per_sm<cdouble>();
template cudaError_t launch_ahq<double>(const int64_t *, const int32_t *, const double *, int64_t, int64_t,
                                        const double *, double *, int, cudaStream_t);
template cudaError_t launch_ahq<cdouble>(const int64_t *, const int32_t *, const cdouble *, int64_t, int64_t,
                                         const cdouble *, cdouble *, int, cudaStream_t);
template cudaError_t launch_spmv_qdot_tiled<double>(const SysView<double> &, int, int64_t, int, const double *,
                                                    double *, double *, double *, int, int *, unsigned *,
                                                    double *, cudaEvent_t, cudaStream_t);
template cudaError_t launch_spmv_qdot_tiled<cdouble>(const SysView<cdouble> &, int, int64_t, int,
                                                     const cdouble *, cdouble *, cdouble *, double *, int, int *,
                                                     unsigned *, double *, cudaEvent_t, cudaStream_t);
template cudaError_t launch_spmv_qdot_tiled<float>(const SysView<float> &, int, int64_t, int, const float *,
                                                   float *, float *, double *, int, int *, unsigned *, double *,
                                                   cudaEvent_t, cudaStream_t);
template cudaError_t launch_spmv_qdot_tiled<cfloat>(const SysView<cfloat> &, int, int64_t, int, const cfloat *,
                                                    cfloat *, cfloat *, double *, int, int *, unsigned *, double *,
                                                    cudaEvent_t, cudaStream_t);
template cudaError_t launch_refine<float, double>(const SysView<float> &, const RefView<double> &,
                                                  const SolveCtl &, const RefCtl &, int, cudaStream_t);
template cudaError_t launch_refine<cfloat, cdouble>(const SysView<cfloat> &, const RefView<cdouble> &,
                                                    const SolveCtl &, const RefCtl &, int, cudaStream_t);
template int refine_blocks_per_sm<float, double>();
template int refine_blocks_per_sm<cfloat, cdouble>();
template cudaError_t launch_batch<double>(const BatchItem<double> *, const BatchPlan &, int, bool, cudaStream_t);
template cudaError_t launch_batch<cdouble>(const BatchItem<cdouble> *, const BatchPlan &, int, bool, cudaStream_t);
template cudaError_t launch_batch_refine<float, double>(const BatchItemR<float, double> *, const BatchPlan &, int,
                                                        bool, cudaStream_t);
template cudaError_t launch_batch_refine<cfloat, cdouble>(const BatchItemR<cfloat, cdouble> *, const BatchPlan &,
                                                          int, bool, cudaStream_t);
template int batch_blocks_per_sm<double>();
template int batch_blocks_per_sm<cdouble>();
template int batch_refine_blocks_per_sm<float, double>();
template int batch_refine_blocks_per_sm<cfloat, cdouble>();

template cudaError_t launch_diag_apply<double>(double *, const double *, int64_t, bool, cudaStream_t);
template cudaError_t launch_diag_apply<cdouble>(cdouble *, const cdouble *, int64_t, bool, cudaStream_t);

}  // namespace mlb
