// Allocation-free fused y = A x, d = Q^H y for callers that cannot
// allocate device memory (see mlbicgstab_spmv_qdot_noalloc in the header).
//
// The per-CTA partial sums live in one fixed array of this library's own
// device memory instead of caller or library allocations.  Every GPU that
// loads the library holds this array until the process exits.
#include <algorithm>
#include <mutex>

#include "../../include/mlbicgstab.h"
#include "mlb_device.cuh"

namespace mlb {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxN = 64;
// Scratch: 256 bytes of header (the CTA ticket counter) followed by the
// per-CTA partial sums, grid * nb * slots doubles.
constexpr int64_t kNaScratchDoubles = 65536;  // 512 KiB
constexpr int64_t kNaHeaderDoubles = 32;       // 256 bytes

static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

// Device address of g_noalloc_scratch, looked up once per device.
std::mutex g_mu;
double *g_addr[256];
bool g_done[256];

int scratch_address(int dev, double **out) {
    if (dev < 0 || dev >= 256) return MLB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_done[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MLB_ERR_CUDA;
        }
        g_addr[dev] = (double *)p;
        g_done[dev] = true;
    }
    *out = g_addr[dev];
    return MLB_OK;
}

__device__ __forceinline__ double ldv(const double *p) { return __ldg(p); }
__device__ __forceinline__ cdouble ldv(const cdouble *p) {
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}

// One thread per CSR row; each thread keeps NB running inner products
// conj(q_k) y over its rows; CTA sums go to the scratch array; the last CTA
// to finish (ticket counter) adds the CTA sums in CTA order and writes d.
template <typename T, int NB>
__global__ void __launch_bounds__(kNaThreads)
    spmv_qdot_csr_kernel(int64_t N, const int64_t *rp, const int32_t *ci, const T *av, const T *x,
                         const T *Q, int64_t ldq, int n, T *y, T *d, double *scratch) {
    constexpr int DS = dslots<T>();
    using ACC = typename real_of<T>::type;
    __shared__ double red[33 * DS];
    __shared__ unsigned s_ticket;
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
    double *part = scratch + kNaHeaderDoubles;
    ACC acc[NB * DS];
#pragma unroll
    for (int k = 0; k < NB * DS; ++k) acc[k] = ACC(0);
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < N;
         row += (int64_t)gridDim.x * blockDim.x) {
        T sum{};
        for (int64_t k = __ldg(rp + row), k1 = __ldg(rp + row + 1); k < k1; ++k)
            sum = efma(ldv(av + k), ldv(x + __ldg(ci + k)), sum);
        y[row] = sum;
#pragma unroll
        for (int q = 0; q < NB; ++q)
            if (q < n) acc_dot(&acc[q * DS], ldv(Q + (int64_t)q * ldq + row), sum);
    }
    // unrolled over the fixed bound NB so that every index into acc is a
    // compile-time constant (a run-time index would put acc in local
    // memory); n is the same in every thread, so the barriers inside
    // block_sum_all are reached uniformly
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (q < n) {
            double v[DS];
#pragma unroll
            for (int t = 0; t < DS; ++t) v[t] = (double)acc[q * DS + t];
            block_sum_all<DS>(v, red);
            if (threadIdx.x == 0) {
#pragma unroll
                for (int t = 0; t < DS; ++t) part[((size_t)blockIdx.x * NB + q) * DS + t] = v[t];
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_ticket = atomicAdd(ticket, 1u);
    }
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();
    for (int q = 0; q < n; ++q) {
        double v[DS];
#pragma unroll
        for (int t = 0; t < DS; ++t) v[t] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
            for (int t = 0; t < DS; ++t) v[t] += part[((size_t)b * NB + q) * DS + t];
        }
        block_sum_all<DS>(v, red);
        if (threadIdx.x == 0) {
            double *dd = reinterpret_cast<double *>(d) + (size_t)q * DS;
#pragma unroll
            for (int t = 0; t < DS; ++t) dd[t] = v[t];
        }
    }
}

template <typename T, int NB>
int launch(int dev, int64_t N, const int64_t *rp, const int32_t *ci, const T *av, const T *x, const T *Q,
           int64_t ldq, int n, T *y, T *d, double *scratch, cudaStream_t st) {
    constexpr int DS = dslots<T>();
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmv_qdot_csr_kernel<T, NB>, kNaThreads, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    int64_t grid = (int64_t)sms * (occ > 0 ? occ : 1);
    const int64_t fit = (kNaScratchDoubles - kNaHeaderDoubles) / ((int64_t)NB * DS);
    const int64_t need = (N + kNaThreads - 1) / kNaThreads;
    grid = std::min(grid, std::min(fit, need));
    if (grid < 1) grid = 1;
    // the ticket counter must start at zero on every call
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), st) != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    spmv_qdot_csr_kernel<T, NB><<<(int)grid, kNaThreads, 0, st>>>(N, rp, ci, av, x, Q, ldq, n, y, d, scratch);
    if (cudaGetLastError() != cudaSuccess) return MLB_ERR_CUDA;
    return MLB_OK;
}

template <typename T>
int dispatch(int dev, int64_t N, const int64_t *rp, const int32_t *ci, const T *av, const T *x, const T *Q,
             int64_t ldq, int n, T *y, T *d, double *scratch, cudaStream_t st) {
    if (n <= 4) return launch<T, 4>(dev, N, rp, ci, av, x, Q, ldq, n, y, d, scratch, st);
    if (n <= 8) return launch<T, 8>(dev, N, rp, ci, av, x, Q, ldq, n, y, d, scratch, st);
    if (n <= 16) return launch<T, 16>(dev, N, rp, ci, av, x, Q, ldq, n, y, d, scratch, st);
    if (n <= 32) return launch<T, 32>(dev, N, rp, ci, av, x, Q, ldq, n, y, d, scratch, st);
    return launch<T, kNaMaxN>(dev, N, rp, ci, av, x, Q, ldq, n, y, d, scratch, st);
}

// Device memory of the current device `dev`, or managed memory.  Memory of
// another GPU is refused: the kernel runs on `dev`, where such a pointer
// is either unmapped (without peer access) or read over NVLink.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace mlb

extern "C" int mlbicgstab_spmv_qdot_noalloc(int64_t nrows, int64_t nnz, const int64_t *row_ptr,
                                            const int32_t *col_idx, const void *values, int32_t dtype,
                                            const void *x, const void *Q, int64_t ldq, int32_t n, void *y,
                                            void *d, void *stream) {
    using namespace mlb;
    if (nrows <= 0 || nrows > (int64_t)INT32_MAX || nnz < 0 || n < 1 || n > kNaMaxN || ldq < nrows)
        return MLB_ERR_ARG;
    if (dtype != MLB_F64 && dtype != MLB_C128) return MLB_ERR_ARG;
    if (!row_ptr || !x || !Q || !y || !d || (nnz > 0 && (!col_idx || !values))) return MLB_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    if (!on_device(row_ptr, dev) || !on_device(x, dev) || !on_device(Q, dev) || !on_device(y, dev) ||
        !on_device(d, dev) || (nnz > 0 && (!on_device(col_idx, dev) || !on_device(values, dev))))
        return MLB_ERR_ARG;
    double *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != MLB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MLB_C128)
        return dispatch<cdouble>(dev, nrows, row_ptr, col_idx, (const cdouble *)values, (const cdouble *)x,
                                 (const cdouble *)Q, ldq, n, (cdouble *)y, (cdouble *)d, scratch, st);
    return dispatch<double>(dev, nrows, row_ptr, col_idx, (const double *)values, (const double *)x,
                            (const double *)Q, ldq, n, (double *)y, (double *)d, scratch, st);
}
