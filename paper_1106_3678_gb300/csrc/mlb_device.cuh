// Device building blocks of the ML(n)BiCGStab library (sm_103a):
// scalar types, 16-byte vector packs, deterministic block/grid reductions
// and a bounded grid barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlb {

// ---------------------------------------------------------------------------
// complex numbers (interleaved re, im; 8- or 16-byte aligned like C99)
// ---------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) cx {
    R re, im;
};

using cdouble = cx<double>;
using cfloat = cx<float>;

template <typename T> struct is_cx { static constexpr bool value = false; };
template <typename R> struct is_cx<cx<R>> { static constexpr bool value = true; };

// Real part type.
template <typename T> struct real_of { using type = T; };
template <typename R> struct real_of<cx<R>> { using type = R; };

// Scalar type of the recurrence coefficients: always FP64 (the small
// coefficient arithmetic stays FP64 even when vectors are FP32).
template <typename T> struct coef_of { using type = double; };
template <typename R> struct coef_of<cx<R>> { using type = cdouble; };

__host__ __device__ __forceinline__ double re_of(double a) { return a; }
__host__ __device__ __forceinline__ double re_of(cdouble a) { return a.re; }
__host__ __device__ __forceinline__ double im_of(double) { return 0.0; }
__host__ __device__ __forceinline__ double im_of(cdouble a) { return a.im; }

__host__ __device__ __forceinline__ cdouble operator+(cdouble a, cdouble b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cdouble operator-(cdouble a, cdouble b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cdouble operator-(cdouble a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cdouble operator*(cdouble a, cdouble b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cdouble operator*(double s, cdouble b) { return {s * b.re, s * b.im}; }
__host__ __device__ __forceinline__ cdouble operator/(cdouble a, cdouble b) {
    double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ cdouble operator/(cdouble a, double s) { return {a.re / s, a.im / s}; }
// FP32 complex (the ILU(0) triangular solves of the refined mode)
__host__ __device__ __forceinline__ cfloat operator-(cfloat a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cfloat operator/(cfloat a, cfloat b) {
    float d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ bool is_zero(double a) { return a == 0.0; }
__host__ __device__ __forceinline__ bool is_zero(cdouble a) { return a.re == 0.0 && a.im == 0.0; }
__host__ __device__ __forceinline__ double abs_of(double a) { return fabs(a); }
__host__ __device__ __forceinline__ double abs_of(cdouble a) { return hypot(a.re, a.im); }
__host__ __device__ __forceinline__ bool finite_of(double a) { return isfinite(a); }
__host__ __device__ __forceinline__ bool finite_of(cdouble a) { return isfinite(a.re) && isfinite(a.im); }
__host__ __device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__host__ __device__ __forceinline__ cdouble recip(cdouble a) { return cdouble{1.0, 0.0} / a; }

// Make a coefficient of compute type T from an FP64 coefficient.
template <typename T> __device__ __forceinline__ T to_t(double a) { return (T)a; }
template <typename T> __device__ __forceinline__ T to_t(cdouble a);
template <> __device__ __forceinline__ cdouble to_t<cdouble>(cdouble a) { return a; }
template <> __device__ __forceinline__ cfloat to_t<cfloat>(cdouble a) { return {(float)a.re, (float)a.im}; }
template <> __device__ __forceinline__ double to_t<double>(double a) { return a; }
template <> __device__ __forceinline__ float to_t<float>(double a) { return (float)a; }

// ---------------------------------------------------------------------------
// element arithmetic: y = a*x + y as fused multiply-adds
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double efma(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ float efma(float a, float x, float y) { return fmaf(a, x, y); }
template <typename R>
__device__ __forceinline__ cx<R> efma(cx<R> a, cx<R> x, cx<R> y) {
    cx<R> o;
    o.re = fmaR(a.re, x.re, fmaR(-a.im, x.im, y.re));
    o.im = fmaR(a.re, x.im, fmaR(a.im, x.re, y.im));
    return o;
}
__device__ __forceinline__ double emul(double a, double x) { return a * x; }
__device__ __forceinline__ float emul(float a, float x) { return a * x; }
template <typename R>
__device__ __forceinline__ cx<R> emul(cx<R> a, cx<R> x) {
    return {fmaR(a.re, x.re, -a.im * x.im), fmaR(a.re, x.im, a.im * x.re)};
}

// Accumulators of inner products: conj(u) v added into acc (re[, im]).
__device__ __forceinline__ void acc_dot(double *a, double u, double v) { a[0] = fma(u, v, a[0]); }
__device__ __forceinline__ void acc_dot(float *a, float u, float v) { a[0] = fmaf(u, v, a[0]); }
template <typename R>
__device__ __forceinline__ void acc_dot(R *a, cx<R> u, cx<R> v) {
    a[0] = fmaR(u.re, v.re, fmaR(u.im, v.im, a[0]));
    a[1] = fmaR(u.re, v.im, fmaR(-u.im, v.re, a[1]));
}
// |v|^2 added into a[0]
__device__ __forceinline__ void acc_nrm(double *a, double v) { a[0] = fma(v, v, a[0]); }
__device__ __forceinline__ void acc_nrm(float *a, float v) { a[0] = fmaf(v, v, a[0]); }
template <typename R>
__device__ __forceinline__ void acc_nrm(R *a, cx<R> v) { a[0] = fmaR(v.re, v.re, fmaR(v.im, v.im, a[0])); }

// Number of accumulator slots one inner product takes.
template <typename T> constexpr int dslots() { return is_cx<T>::value ? 2 : 1; }

// ---------------------------------------------------------------------------
// 16-byte packs of vector elements
// ---------------------------------------------------------------------------
template <typename T>
struct alignas(16) Pack {
    static constexpr int W = 16 / sizeof(T);
    T e[W];
};

template <typename T>
__device__ __forceinline__ Pack<T> ldp(const T *base, int64_t c) {
    // coherent load (data may have been written earlier in the same launch)
    uint4 u = reinterpret_cast<const uint4 *>(base)[c];
    Pack<T> p;
    *reinterpret_cast<uint4 *>(&p) = u;
    return p;
}
template <typename T>
__device__ __forceinline__ Pack<T> ldp_ro(const T *base, int64_t c) {
    // read-only for the lifetime of the kernel (Q, F, matrix)
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(base) + c);
    Pack<T> p;
    *reinterpret_cast<uint4 *>(&p) = u;
    return p;
}
template <typename T>
__device__ __forceinline__ void stp(T *base, int64_t c, const Pack<T> &p) {
    reinterpret_cast<uint4 *>(base)[c] = *reinterpret_cast<const uint4 *>(&p);
}

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void warp_sum(double (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Sum K values over the CTA; every thread receives the totals.  `red` is
// shared scratch of at least 33*K doubles.  Fixed order: deterministic.
template <int K>
__device__ __forceinline__ void block_sum_all(double (&v)[K], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    warp_sum<K>(v);
    __syncthreads();  // red may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = lane < nw ? red[k * 32 + lane] : 0.0;
        warp_sum<K>(t);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) red[32 * K + k] = t[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[32 * K + k];
}

// ---------------------------------------------------------------------------
// memory-model helpers and the bounded grid barrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Barrier state in global memory (zeroed before every launch).
struct BarrierState {
    unsigned count;   // arrivals since the launch began (monotonic)
    unsigned pad0;
    int status;       // 0, or an MLB_ERR_* code set by a CTA that gave up
    int pad1;
};

constexpr int kStatusTimeout = 4;  // == MLB_ERR_TIMEOUT

// Arrive-and-wait of one CTA, executed by thread 0 only, after the CTA's
// writes have been ordered before it (a __syncthreads, or thread 0's own
// writes).  `epoch` counts the barriers this CTA has passed; all CTAs pass
// the same sequence, so barrier e completes when the counter reaches
// e * expected.  The spin is bounded by timeout_ns (%globaltimer) and
// gives up early when another CTA has already recorded a failure.
// grid_arrive and grid_wait are its two halves, for callers with work to
// overlap with the wait.
__device__ __forceinline__ void grid_arrive(BarrierState *bs, unsigned &epoch) {
    epoch += 1;
    red_release_add_u32(&bs->count, 1u);
}
__device__ __forceinline__ bool grid_wait(BarrierState *bs, unsigned epoch, unsigned expected,
                                          uint64_t timeout_ns) {
    const unsigned target = epoch * expected;
    uint64_t t0 = 0;
    unsigned spins = 0;
    while ((int)(ld_acquire_u32(&bs->count) - target) < 0) {
        if ((++spins & 31u) == 0) {
            if (ld_relaxed_i32(&bs->status) != 0) return false;
            const uint64_t t = globaltimer_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > timeout_ns) {
                atomicCAS(&bs->status, 0, kStatusTimeout);
                return false;
            }
        }
        __nanosleep(16);
    }
    fence_acq_rel_gpu();
    return true;
}
__device__ __forceinline__ bool grid_arrive_wait(BarrierState *bs, unsigned &epoch, unsigned expected,
                                                 uint64_t timeout_ns) {
    grid_arrive(bs, epoch);
    return grid_wait(bs, epoch, expected, timeout_ns);
}

// Whole-CTA grid barrier: every thread calls it; returns false (uniformly
// in the CTA) when the wait failed, and the caller must then return.
__device__ __forceinline__ bool grid_barrier(BarrierState *bs, unsigned &epoch, unsigned expected,
                                             uint64_t timeout_ns, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = grid_arrive_wait(bs, epoch, expected, timeout_ns) ? 1 : 0;
    __syncthreads();
    return *s_flag != 0;
}

}  // namespace mlb
