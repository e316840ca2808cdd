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
constexpr int kStageBytes = 40 * 1024;              // 160 KB of stages
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
};

__device__ __forceinline__ void ring_init(TileRing *R, unsigned char *buf) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&R->full[s], 1);
            mbar_init(&R->empty[s], kConsumerWarps);
        }
        R->buf = buf;
        R->failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Dynamic shared memory a kernel needs for the ring (plus alignment slack).
constexpr size_t kRingBytes = (size_t)kStages * kStageBytes + 128;

__device__ __forceinline__ unsigned char *ring_buffer(unsigned char *dsm) {
    return (unsigned char *)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
}

// A streaming pass over the chunk range [c_lo, c_hi) of this CTA: `ni`
// inputs of 16-byte chunks, tiles of `tc` chunks per input.
struct TilePass {
    const void *in[kMaxInputs];
    int ni;
    int tc;
    int64_t c_lo, c_hi;
    __device__ __forceinline__ int ntiles() const { return (int)((c_hi - c_lo + tc - 1) / tc); }
};

__device__ __forceinline__ int tile_chunks_for(int ni) {
    int tc = kStageBytes / (16 * ni);
    if (tc > kTileChunks) tc = kTileChunks;
    return tc & ~31;   // whole warps of chunks
}

// Producer side (lane 0 of the producer warp): issue every tile of pass P.
// `seq` is this CTA's running tile sequence number.
__device__ __forceinline__ bool produce(TileRing *R, const TilePass &P, unsigned &seq, uint64_t timeout_ns) {
    const int nt = P.ntiles();
    for (int t = 0; t < nt; ++t, ++seq) {
        const int s = (int)(seq % kStages);
        const unsigned use = seq / kStages;
        if (use > 0 && !mbar_wait(&R->empty[s], (use - 1) & 1u, timeout_ns)) return false;
        const int64_t c0 = P.c_lo + (int64_t)t * P.tc;
        int64_t cn = P.c_hi - c0;
        if (cn > P.tc) cn = P.tc;
        const unsigned bytes = (unsigned)(cn * 16);
        mbar_arrive_expect_tx(&R->full[s], bytes * (unsigned)P.ni);
        unsigned char *dst = R->buf + (size_t)s * kStageBytes;
        for (int i = 0; i < P.ni; ++i)
            bulk_g2s(dst + (size_t)i * P.tc * 16, (const unsigned char *)P.in[i] + c0 * 16, bytes, &R->full[s]);
    }
    return true;
}

// Consumer side: for every tile, wait for it, call fn(chunk, stage, k)
// for each chunk k of the tile owned by this thread (chunk k is read from
// stage + i*tc*16 + k*16 for input i), then release the stage.
template <typename Fn>
__device__ __forceinline__ bool consume(TileRing *R, const TilePass &P, unsigned &seq, uint64_t timeout_ns, Fn fn) {
    const int nt = P.ntiles();
    const int tid = threadIdx.x;   // < kConsumers
    for (int t = 0; t < nt; ++t, ++seq) {
        const int s = (int)(seq % kStages);
        const unsigned use = seq / kStages;
        if (!mbar_wait(&R->full[s], use & 1u, timeout_ns)) return false;
        const int64_t c0 = P.c_lo + (int64_t)t * P.tc;
        int64_t cn = P.c_hi - c0;
        if (cn > P.tc) cn = P.tc;
        const unsigned char *stage = R->buf + (size_t)s * kStageBytes;
        for (int k = tid; k < cn; k += kConsumers) fn(c0 + k, stage, k);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&R->empty[s]);
    }
    fence_proxy_async_global();
    return true;
}

// SELL-32 tiles: `spt` consecutive slices [s0, s0+spt) of this CTA's slice
// range; the stage holds their values (first) and column indices.
__device__ __forceinline__ bool produce_sell(TileRing *R, int64_t s_lo, int64_t s_hi, int spt,
                                             const int64_t *slice_ptr, const void *sval, int vbytes,
                                             const int32_t *scol, unsigned &seq, uint64_t timeout_ns) {
    for (int64_t s0 = s_lo; s0 < s_hi; s0 += spt, ++seq) {
        const int s = (int)(seq % kStages);
        const unsigned use = seq / kStages;
        if (use > 0 && !mbar_wait(&R->empty[s], (use - 1) & 1u, timeout_ns)) return false;
        const int64_t s1 = s0 + spt < s_hi ? s0 + spt : s_hi;
        const int64_t e0 = __ldg(slice_ptr + s0), e1 = __ldg(slice_ptr + s1);
        const unsigned nv = (unsigned)(e1 - e0);
        const unsigned bv = nv * (unsigned)vbytes, bc = nv * 4u;
        mbar_arrive_expect_tx(&R->full[s], bv + bc);
        unsigned char *dst = R->buf + (size_t)s * kStageBytes;
        if (nv > 0) {
            bulk_g2s(dst, (const unsigned char *)sval + e0 * vbytes, bv, &R->full[s]);
            bulk_g2s(dst + bv, scol + e0, bc, &R->full[s]);
        }
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
