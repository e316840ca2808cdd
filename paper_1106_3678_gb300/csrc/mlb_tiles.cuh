// Shared-memory tile pipeline fed by TMA bulk copies (cp.async.bulk) for
// the streaming passes of the solve engine.
//
// One producer warp (the last warp of the CTA) copies tiles of every input
// vector of a pass from global memory into a ring of shared-memory stages;
// the consumer warps compute from shared memory and store their outputs to
// global memory directly.  Loads therefore run ahead of the FP64
// arithmetic instead of alternating with it.  Each stage has a "full"
// mbarrier (transaction count of the bulk copies) and an "empty" mbarrier
// (one arrival per consumer warp).  Every wait is bounded.
//
// A CTA only ever bulk-loads vector ranges it owns (or read-only data), and
// a pass never bulk-loads what the same pass writes.  So the only
// cross-proxy ordering needed is CTA-local and per pass: each consumer
// thread fences its generic-proxy stores with fence.proxy.async once at the
// end of a pass, before the CTA barrier after which the producer may issue
// bulk copies of that data.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlb_device.cuh"

namespace mlb {

constexpr int kConsumerWarps = 15;                  // 480 consumer threads
constexpr int kConsumers = 32 * kConsumerWarps;
constexpr int kTileThreads = kConsumers + 32;       // + one producer warp
constexpr int kStages = 4;
constexpr int kStageBytes = 44 * 1024;              // 176 KB of stages
constexpr int kTileChunks = kConsumers;             // 16-byte chunks per input per tile (max)
constexpr int kMaxInputs = 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with parity `phase` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned phase, uint64_t timeout_ns) {
    if (mbar_test(b, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(b, phase)) return true;
        if ((it & 15u) == 0 && globaltimer_ns() - t0 > timeout_ns) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Bulk copy with an L2 eviction-priority hint (for data streamed once).
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Ring state of one CTA (in shared memory; producer and consumers advance
// their own sequence counters in lock step over the same tiles).
struct TileRing {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    unsigned char *buf;      // kStages * kStageBytes, 128-byte aligned
    unsigned issued;         // tiles issued (producer lane 0 only)
    unsigned consumed;       // tiles consumed (every consumer thread, uniform)
    int failed;              // set when a wait timed out
    // Cache of the SELL-32 slice offsets of this CTA's slice range:
    // soff[i] = slice_ptr[soff_lo + i] - soff_base for i = 0..soff_hi-soff_lo
    // (kept in the dynamic shared memory after the stages).
    int32_t *soff;
    const int64_t *soff_src; // slice_ptr the cache was filled from (null: empty)
    int64_t soff_lo, soff_hi, soff_base;
};

__device__ __forceinline__ void ring_init(TileRing *R, unsigned char *buf) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&R->full[s], 1);
            mbar_init(&R->empty[s], kConsumerWarps);
        }
        R->buf = buf;
        R->failed = 0;
        R->soff = reinterpret_cast<int32_t *>(buf + (size_t)kStages * kStageBytes);
        R->soff_src = nullptr;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Slice offsets cached per CTA (slices of one CTA's share, plus one).
constexpr int kSoffCap = 2048;

// Dynamic shared memory a kernel needs for the ring and the offset cache
// (plus alignment slack).
constexpr size_t kRingBytes = (size_t)kStages * kStageBytes + (size_t)kSoffCap * 4 + 128;

// Fill the slice-offset cache for slices [s_lo, s_hi] (all threads of the
// CTA call this).  The cache stays empty when the range has more than
// kSoffCap - 1 slices or spans 2^31 or more entries; SpMV passes then read
// slice_ptr from global memory.
__device__ __forceinline__ void soff_load(TileRing *R, const int64_t *slice_ptr, int64_t s_lo, int64_t s_hi) {
    __syncthreads();   // no thread still reads an earlier cache
    const int64_t n = s_hi - s_lo;
    const int64_t base = __ldg(slice_ptr + s_lo);
    const bool fits = n + 1 <= kSoffCap && __ldg(slice_ptr + s_hi) - base < ((int64_t)1 << 31);
    if (fits)
        for (int64_t i = threadIdx.x; i <= n; i += blockDim.x)
            R->soff[i] = (int32_t)(__ldg(slice_ptr + s_lo + i) - base);
    if (threadIdx.x == 0) {
        R->soff_src = fits ? slice_ptr : nullptr;
        R->soff_lo = s_lo;
        R->soff_hi = s_hi;
        R->soff_base = base;
    }
    __syncthreads();
}

// Offset source of one SpMV pass over slices [s_lo, s_hi): the cache when
// it holds that range of that matrix, else global memory.
struct SliceOffsets {
    const int32_t *so;       // cache, or null
    const int64_t *sp;       // slice_ptr
    int64_t lo, base;
    __device__ __forceinline__ SliceOffsets(const TileRing *R, const int64_t *slice_ptr, int64_t s_lo, int64_t s_hi)
        : so(nullptr), sp(slice_ptr), lo(s_lo), base(0) {
        if (R->soff_src == slice_ptr && R->soff_lo == s_lo && R->soff_hi == s_hi) {
            so = R->soff;
            base = R->soff_base;
        }
    }
    // slice_ptr[s] for s in [lo, hi]
    __device__ __forceinline__ int64_t operator()(int64_t s) const {
        return so ? base + so[s - lo] : __ldg(sp + s);
    }
};

__device__ __forceinline__ unsigned char *ring_buffer(unsigned char *dsm) {
    return (unsigned char *)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
}

// The producer lane's copy descriptor of a streaming pass over the chunk
// range [c_lo, c_hi) of this CTA: `ni` inputs of 16-byte chunks, tiles of
// `tc` chunks per input.
struct TilePass {
    const void *in[kMaxInputs];
    int ni;
    int tc;
    int64_t c_lo, c_hi;
};

// Geometry of a streaming pass as the consumers see it: chunks per tile
// and the CTA's chunk range.
struct TileGeom {
    int tc;
    int64_t c_lo, c_hi;
};

__device__ __forceinline__ int tile_chunks_for(int ni) {
    int tc = kStageBytes / (16 * ni);
    if (tc > kTileChunks) tc = kTileChunks;
    return tc & ~31;   // whole warps of chunks
}

// Producer side (lane 0 of the producer warp): issue every tile of pass P.
// `seq` is this CTA's running tile sequence number.
__device__ __forceinline__ bool produce(TileRing *R, const TilePass &P, unsigned &seq, uint64_t timeout_ns) {
    // The descriptor lives in memory (its input list is indexed at run
    // time); copy it into registers once, so the issue loop does not wait
    // on a load before every copy.
    const unsigned char *src[kMaxInputs];
#pragma unroll
    for (int i = 0; i < kMaxInputs; ++i) src[i] = i < P.ni ? (const unsigned char *)P.in[i] : nullptr;
    const int ni = P.ni, tc = P.tc;
    const int64_t c_lo = P.c_lo, c_hi = P.c_hi;
    unsigned char *const buf = R->buf;
    const int nt = (int)((c_hi - c_lo + tc - 1) / tc);
    for (int t = 0; t < nt; ++t, ++seq) {
        const int s = (int)(seq % kStages);
        const unsigned use = seq / kStages;
        if (use > 0 && !mbar_wait(&R->empty[s], (use - 1) & 1u, timeout_ns)) return false;
        const int64_t c0 = c_lo + (int64_t)t * tc;
        int64_t cn = c_hi - c0;
        if (cn > tc) cn = tc;
        const unsigned bytes = (unsigned)(cn * 16);
        mbar_arrive_expect_tx(&R->full[s], bytes * (unsigned)ni);
        unsigned char *dst = buf + (size_t)s * kStageBytes;
#pragma unroll
        for (int i = 0; i < kMaxInputs; ++i)
            if (i < ni) bulk_g2s(dst + (size_t)i * tc * 16, src[i] + c0 * 16, bytes, &R->full[s]);
    }
    return true;
}

// Consumer side: for every tile, wait for it, call fn(chunk, stage, k)
// for each chunk k of the tile owned by this thread (chunk k is read from
// stage + i*tc*16 + k*16 for input i), then release the stage.
template <typename Fn>
__device__ __forceinline__ bool consume(TileRing *R, const TileGeom g, unsigned &seq, uint64_t timeout_ns, Fn fn) {
    const int tc = g.tc;
    const int64_t c_lo = g.c_lo, c_hi = g.c_hi;
    const int nt = (int)((c_hi - c_lo + tc - 1) / tc);
    unsigned char *const buf = R->buf;
    unsigned sq = seq;
    const int tid = threadIdx.x;   // < kConsumers
    for (int t = 0; t < nt; ++t, ++sq) {
        const int s = (int)(sq % kStages);
        const unsigned use = sq / kStages;
        if (!mbar_wait(&R->full[s], use & 1u, timeout_ns)) {
            seq = sq;
            return false;
        }
        const int64_t c0 = c_lo + (int64_t)t * tc;
        int64_t cn = c_hi - c0;
        if (cn > tc) cn = tc;
        const unsigned char *stage = buf + (size_t)s * kStageBytes;
        for (int k = tid; k < cn; k += kConsumers) fn(c0 + k, stage, k);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&R->empty[s]);
    }
    seq = sq;
    fence_proxy_async_global();
    return true;
}

// SELL-32 tiles: `spt` consecutive slices [s0, s0+spt) of this CTA's slice
// range.  A stage holds their values (vbytes per entry: one value, or the
// three of a 3x3-block entry), then their column indices, then for each of
// the `ne` epilogue vectors the 32*spt entries (ebytes each) of the tile's
// rows (those rows belong to this CTA).  The matrix is streamed once per
// product, so its copies carry an L2 evict-first hint.
__device__ __forceinline__ bool produce_sell(TileRing *R, int64_t s_lo, int64_t s_hi, int spt,
                                             const SliceOffsets &off, const void *sval, int vbytes, int ebytes,
                                             const int32_t *scol, const void *const *epi, int ne,
                                             unsigned &seq, uint64_t timeout_ns) {
    const uint64_t pol = l2_evict_first_policy();
    for (int64_t s0 = s_lo; s0 < s_hi; s0 += spt, ++seq) {
        const int s = (int)(seq % kStages);
        const unsigned use = seq / kStages;
        if (use > 0 && !mbar_wait(&R->empty[s], (use - 1) & 1u, timeout_ns)) return false;
        const int64_t s1 = s0 + spt < s_hi ? s0 + spt : s_hi;
        const int64_t e0 = off(s0), e1 = off(s1);
        const unsigned nv = (unsigned)(e1 - e0);
        const unsigned bv = nv * (unsigned)vbytes, bc = nv * 4u;
        const unsigned be = (unsigned)(s1 - s0) * 32u * (unsigned)ebytes;
        mbar_arrive_expect_tx(&R->full[s], bv + bc + be * (unsigned)ne);
        unsigned char *dst = R->buf + (size_t)s * kStageBytes;
        if (nv > 0) {
            bulk_g2s_hint(dst, (const unsigned char *)sval + e0 * vbytes, bv, &R->full[s], pol);
            bulk_g2s_hint(dst + bv, scol + e0, bc, &R->full[s], pol);
        }
        unsigned char *de = dst + bv + bc;
        for (int i = 0; i < ne; ++i)
            bulk_g2s(de + (size_t)i * spt * 32 * ebytes, (const unsigned char *)epi[i] + s0 * 32 * ebytes, be,
                     &R->full[s]);
    }
    return true;
}

// At the end of a kernel: wait (bounded) until every tile the producer
// issued has landed, so that no bulk copy is still writing into shared
// memory when the CTA exits.  In normal operation every issued tile has
// already been consumed and this returns at once.
__device__ __forceinline__ void ring_drain(TileRing *R, unsigned pseq, unsigned cseq, uint64_t timeout_ns) {
    if ((threadIdx.x >> 5) == kConsumerWarps && (threadIdx.x & 31) == 0) R->issued = pseq;
    if (threadIdx.x == 0) R->consumed = cseq;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (unsigned q = R->consumed; q < R->issued; ++q)
            if (!mbar_wait(&R->full[q % kStages], (q / kStages) & 1u, timeout_ns)) break;
    }
    __syncthreads();
}

}  // namespace mlb
