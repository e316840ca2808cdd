// C ABI of the ML(n)BiCGStab library: argument validation, device state of
// a handle, and the host side of every entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/mlbicgstab.h"
#include "mlb_internal.h"

using namespace mlb;

struct mlb_handle {
    int dtype = MLB_F64;
    int n = 4;          // shadow vectors Q and F were built for
    int n_active = 4;   // shadow vectors the next solve uses (<= n)
    int precond = MLB_PRECOND_NONE;
    void *mdiag = nullptr;   // diagonal of M (Jacobi), device, N values
    // multicolour ILU(0): the handle holds P A P^T; perm[new] = old row
    std::vector<int32_t> perm_h;
    int32_t *perm_d = nullptr;
    void *pstage = nullptr;   // device staging vector for the reordering
    int ncolors = 0;
    // ILU(0) factors and level sets (device; see IluHost)
    int64_t *ilu_rp = nullptr;
    int32_t *ilu_ci = nullptr, *ilu_dpos = nullptr;
    int32_t *ilu_lrows = nullptr, *ilu_lptr = nullptr, *ilu_urows = nullptr, *ilu_uptr = nullptr;
    void *ilu_lu = nullptr, *ilu_t = nullptr;
    int ilu_nlev_l = 0, ilu_nlev_u = 0;
    int64_t ilu_nnz = 0;
    int32_t *ilu_lcnt = nullptr, *ilu_ucnt = nullptr, *ilu_lell_c = nullptr, *ilu_uell_c = nullptr;
    void *ilu_lell_a = nullptr, *ilu_uell_a = nullptr, *ilu_udiag = nullptr;
    // refined mode with ILU(0): FP32 copies of the factor values and an
    // FP32 work vector for M^{-1}
    void *ilu_lu32 = nullptr, *ilu_t32 = nullptr, *ilu_lell_a32 = nullptr, *ilu_uell_a32 = nullptr,
         *ilu_udiag32 = nullptr;
    int precision = MLB_PREC_FP64;
    int64_t N = 0, ld = 0, nnz = 0, nnz_pad = 0, nslices = 0;
    int64_t maxw = 0;   // widest SELL-32 slice (entries per row)
    int ew = 1;         // values per stored entry: 1, or 3 (3x3-block rows, one column per three values)
    int device = 0;
    cudaStream_t stream = nullptr;
    int grid = 1;
    int grid_max = 1;       // largest co-resident grid of the solve kernel
    int grid_want = 1;      // CTAs that give every CTA at least 512 chunks
    int spt_cap = kConsumerWarps;   // cap on slices per SpMV tile (autotuner)
    int batch_spt = -1;   // the same in batches (batch autotuner; -1: spt_cap)
    int batch_team = 4;   // CTAs per team for a batch's large systems (1: none)
    int qd_ne = 0;        // columns fused into the product's epilogue (autotuner; 0: built-in rule)
    uint64_t timeout_ns = 2000000000ull;
    double kappa = 0.0;
    int max_outer = 10;
    double inner_tol = 1e-2;
    int64_t inner_maxit = 1000000;
    size_t esize = 8;  // bytes per value
    // device buffers
    int64_t *slice_ptr = nullptr;
    int32_t *scol = nullptr;
    void *sval = nullptr;
    void *Q = nullptr, *F = nullptr, *G = nullptr, *W = nullptr;
    void *x = nullptr, *r = nullptr, *z = nullptr, *b = nullptr;
    // refined mode: FP32 copies of the matrix values, Q, F and the inner
    // solver's vectors (x, r, b above stay FP64: solution, true residual,
    // right-hand side)
    void *sval32 = nullptr, *Q32 = nullptr, *F32 = nullptr, *G32 = nullptr, *W32 = nullptr;
    void *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *b32 = nullptr;
    void *xbest = nullptr;   // refined mode: best FP64 solution so far
    double *partials = nullptr;
    BarrierState *bar = nullptr;
    DevResult *dres = nullptr;
    double *err_hist = nullptr;
    int64_t err_cap = 0;
    double *qd_partials = nullptr;
    double *qd_out = nullptr;
    int *qd_status = nullptr;     // one slot per CTA of the fused product
    unsigned *qd_ticket = nullptr;  // last-CTA counter, 0 between launches
    double qd_ms = 0.0;           // device time of the last fused product
    double *qd_host = nullptr;    // pinned copy of qd_out
    DevResult *hres = nullptr;  // pinned
    // batch workspace (owned by the first handle of a batch call)
    void *bws = nullptr;
    size_t bws_bytes = 0;
    void *bhost = nullptr;      // pinned staging of items and results
    size_t bhost_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
};

namespace {

#define MLB_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            return e_ == cudaErrorMemoryAllocation ? MLB_ERR_OOM : MLB_ERR_CUDA; \
        }                                                                       \
    } while (0)

int dev_alloc(mlb_handle *h, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? MLB_ERR_OOM : MLB_ERR_CUDA;
    }
    h->allocs.push_back(*p);
    h->device_bytes += (int64_t)bytes;
    return MLB_OK;
}

template <typename P>
int dev_alloc_t(mlb_handle *h, P **p, size_t bytes) {
    void *v = nullptr;
    int rc = dev_alloc(h, &v, bytes);
    *p = (P *)v;
    return rc;
}

// CSR checks done before any GPU work.
int validate_csr(const mlb_matrix *A) {
    if (!A || A->nrows <= 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->values)))
        return MLB_ERR_ARG;
    if (A->dtype != MLB_F64 && A->dtype != MLB_C128) return MLB_ERR_ARG;
    if (A->block != 0 && A->block != 1 && A->block != 3) return MLB_ERR_ARG;
    if (A->nrows > (int64_t)INT32_MAX - 1024) return MLB_ERR_ARG;
    const int64_t bs = A->block == 3 ? 3 : 1;
    if (A->nrows % bs != 0) return MLB_ERR_ARG;
    const int64_t nb = A->nrows / bs;   // (block) rows of row_ptr
    if (A->row_ptr[0] != 0 || A->row_ptr[nb] != A->nnz) return MLB_ERR_ARG;
    for (int64_t r = 0; r < nb; ++r)
        if (A->row_ptr[r + 1] < A->row_ptr[r]) return MLB_ERR_ARG;
    for (int64_t k = 0; k < A->nnz; ++k)
        if (A->col_idx[k] < 0 || (int64_t)A->col_idx[k] >= nb) return MLB_ERR_ARG;
    return MLB_OK;
}

// BSR with 3x3 blocks (block = 3) as scalar CSR: row 3R + a lists, block
// by block in the given order, the three values of row a of each block
// with columns 3C, 3C+1, 3C+2.
void bsr3_expand(const mlb_matrix *A, size_t es, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                 std::vector<char> &val) {
    const int64_t nb = A->nrows / 3;
    rp.assign(A->nrows + 1, 0);
    for (int64_t R = 0; R < nb; ++R)
        for (int a = 0; a < 3; ++a)
            rp[3 * R + a + 1] = rp[3 * R + a] + 3 * (A->row_ptr[R + 1] - A->row_ptr[R]);
    ci.assign(rp[A->nrows], 0);
    val.assign((size_t)rp[A->nrows] * es, 0);
    const char *av = (const char *)A->values;
    for (int64_t R = 0; R < nb; ++R)
        for (int a = 0; a < 3; ++a) {
            int64_t d = rp[3 * R + a];
            for (int64_t k = A->row_ptr[R]; k < A->row_ptr[R + 1]; ++k)
                for (int j = 0; j < 3; ++j, ++d) {
                    ci[d] = 3 * A->col_idx[k] + j;
                    memcpy(&val[(size_t)d * es], av + ((size_t)k * 9 + a * 3 + j) * es, es);
                }
        }
}

// Every row's entries come in groups of three consecutive columns 3C,
// 3C+1, 3C+2 (a matrix of 3x3 blocks, stored row by row): the products
// can then keep one column index per three values.
bool has_triplets(const mlb_matrix *A) {
    if (A->nrows % 3 != 0) return false;
    for (int64_t r = 0; r < A->nrows; ++r) {
        const int64_t k0 = A->row_ptr[r], k1 = A->row_ptr[r + 1];
        if ((k1 - k0) % 3 != 0) return false;
        for (int64_t k = k0; k < k1; k += 3)
            if (A->col_idx[k] % 3 != 0 || A->col_idx[k + 1] != A->col_idx[k] + 1 ||
                A->col_idx[k + 2] != A->col_idx[k] + 2)
                return false;
    }
    return true;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// CSR -> SELL-32 (slices of 32 consecutive rows, natural row order, entry k
// of lane l at slice_ptr[s] + 32k + l; padding entries have value 0 and
// column = the row itself, clamped to N-1).
// ew = 3 (a matrix with has_triplets): each stored entry is three values
// of one row of a 3x3 block and the block's first column; entry k of lane
// l holds its values at 3 (slice_ptr[s] + 32k + l) .. + 2.  Padding entries
// have value(s) 0 and a column whose entries (c .. c + ew - 1) exist.
int64_t csr_to_sell32(const mlb_matrix *A, int64_t ld, std::vector<int64_t> &sp, std::vector<int32_t> &col,
                      std::vector<char> &val, size_t es, int ew) {
    const int64_t N = A->nrows, ns = ld / 32;
    sp.assign(ns + 1, 0);
    int64_t maxw = 0;
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t l = 0; l < 32; ++l) {
            int64_t row = s * 32 + l;
            if (row < N) w = std::max(w, (A->row_ptr[row + 1] - A->row_ptr[row]) / ew);
        }
        sp[s + 1] = sp[s] + 32 * w;
        maxw = std::max(maxw, w);
    }
    const int64_t tot = sp[ns];
    col.assign(tot, 0);
    val.assign(tot * es * ew, 0);
    const char *av = (const char *)A->values;
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t w = (sp[s + 1] - sp[s]) / 32;
        for (int64_t l = 0; l < 32; ++l) {
            const int64_t row = s * 32 + l;
            const int64_t len = row < N ? (A->row_ptr[row + 1] - A->row_ptr[row]) / ew : 0;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t dst = sp[s] + 32 * k + l;
                if (k < len) {
                    const int64_t src = A->row_ptr[row] + ew * k;
                    col[dst] = A->col_idx[src];
                    memcpy(&val[dst * es * ew], av + src * es, es * ew);
                } else {
                    const int64_t r = std::min<int64_t>(row, N - 1);
                    col[dst] = (int32_t)(ew == 3 ? r - r % 3 : r);
                }
            }
        }
    }
    return maxw;
}

// Slices per SpMV tile so that the widest tile (entries of `ew` values of
// `vbytes` plus a 4-byte column index, and `nepi` epilogue vectors) fits
// one shared-memory stage; 0 when one slice alone does not fit (the SpMV
// then reads the matrix directly).
int slices_per_tile(int64_t maxw, size_t vbytes, int nepi, int ew = 1) {
    const int64_t per_slice = maxw * 32 * (int64_t)(ew * vbytes + 4) + (int64_t)nepi * 32 * (int64_t)vbytes;
    if (per_slice <= 0) return kConsumerWarps;
    int64_t spt = kStageBytes / per_slice;
    if (spt > kConsumerWarps) spt = kConsumerWarps;
    return (int)spt;
}
void set_spt(int (&spt)[3], int64_t maxw, size_t vbytes, int cap, int ew) {
    for (int e = 0; e < 3; ++e) spt[e] = std::min(slices_per_tile(maxw, vbytes, e, ew), cap);
}

// A^H in CSR by a stable counting sort over columns (values conjugated for
// complex data).
void conj_transpose(const mlb_matrix *A, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                    std::vector<char> &av, size_t es, bool cplx) {
    const int64_t N = A->nrows, nnz = A->nnz;
    rp.assign(N + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) rp[A->col_idx[k] + 1]++;
    for (int64_t r = 0; r < N; ++r) rp[r + 1] += rp[r];
    std::vector<int64_t> next(rp.begin(), rp.end() - 1);
    ci.assign(nnz, 0);
    av.assign(nnz * es, 0);
    const char *src = (const char *)A->values;
    for (int64_t r = 0; r < N; ++r) {
        for (int64_t k = A->row_ptr[r]; k < A->row_ptr[r + 1]; ++k) {
            const int64_t dst = next[A->col_idx[k]]++;
            ci[dst] = (int32_t)r;
            memcpy(&av[dst * es], src + k * es, es);
            if (cplx) {
                double *im = (double *)&av[dst * es] + 1;
                *im = -*im;
            }
        }
    }
}

// Cap on slices per SpMV tile inside a batch: the batch autotuner's
// choice, else the handle's own.
int batch_cap(const mlb_handle *h) { return h->batch_spt >= 0 ? h->batch_spt : h->spt_cap; }

// Columns of Q fused into the fused product's epilogue: the autotuner's
// choice while the active n allows it, else the built-in rule for the
// product's value type (narrow: the FP32 copies).
int qd_ne_for(const mlb_handle *h, bool cplx, bool narrow) {
    const int n = h->n_active, t = h->qd_ne;
    if ((t == 1 || t == 2 || (t == 4 && !cplx)) && t <= n) return t;
    return qd_fused_columns(n, cplx, narrow);
}

// The handle applies ILU(0) factors (natural or multicolour order).
bool has_ilu(const mlb_handle *h) {
    return h->precond == MLB_PRECOND_ILU0 || h->precond == MLB_PRECOND_ILU0_MC;
}

template <typename T>
SysView<T> make_view(const mlb_handle *h) {
    SysView<T> v;
    v.N = h->N;
    v.ld = h->ld;
    v.nnz = h->nnz;
    v.nslices = h->nslices;
    v.slice_ptr = h->slice_ptr;
    v.scol = h->scol;
    v.sval = (const T *)h->sval;
    set_spt(v.spt, h->maxw, sizeof(T), h->spt_cap, h->ew);
    v.ew = h->ew;
    v.narrow_rows = h->maxw <= 7 ? 1 : 0;
    v.Q = (const T *)h->Q;
    v.F = (const T *)h->F;
    v.G = (T *)h->G;
    v.W = (T *)h->W;
    v.x = (T *)h->x;
    v.r = (T *)h->r;
    v.z = (T *)h->z;
    v.b = (T *)h->b;
    v.n = h->n_active;
    v.ilu = IluView<T>{};
    if (has_ilu(h)) {
        v.ilu.rp = h->ilu_rp;
        v.ilu.ci = h->ilu_ci;
        v.ilu.lu = (const T *)h->ilu_lu;
        v.ilu.dpos = h->ilu_dpos;
        v.ilu.lrows = h->ilu_lrows;
        v.ilu.lptr = h->ilu_lptr;
        v.ilu.urows = h->ilu_urows;
        v.ilu.uptr = h->ilu_uptr;
        v.ilu.nlev_l = h->ilu_nlev_l;
        v.ilu.nlev_u = h->ilu_nlev_u;
        v.ilu.nnz = h->ilu_nnz;
        v.ilu.t = (T *)h->ilu_t;
        v.ilu.lcnt = h->ilu_lcnt;
        v.ilu.ucnt = h->ilu_ucnt;
        v.ilu.lell_c = h->ilu_lell_c;
        v.ilu.uell_c = h->ilu_uell_c;
        v.ilu.lell_a = (const T *)h->ilu_lell_a;
        v.ilu.uell_a = (const T *)h->ilu_uell_a;
        v.ilu.udiag = (const T *)h->ilu_udiag;
    }
    return v;
}

template <typename T32>
SysView<T32> make_view32(const mlb_handle *h) {
    SysView<T32> v;
    v.N = h->N;
    v.ld = h->ld;
    v.nnz = h->nnz;
    v.nslices = h->nslices;
    v.slice_ptr = h->slice_ptr;
    v.scol = h->scol;
    v.sval = (const T32 *)h->sval32;
    set_spt(v.spt, h->maxw, sizeof(T32), h->spt_cap, h->ew);
    v.ew = h->ew;
    v.narrow_rows = h->maxw <= 7 ? 1 : 0;
    v.Q = (const T32 *)h->Q32;
    v.F = (const T32 *)h->F32;
    v.G = (T32 *)h->G32;
    v.W = (T32 *)h->W32;
    v.x = (T32 *)h->x32;
    v.r = (T32 *)h->r32;
    v.z = (T32 *)h->z32;
    v.b = (T32 *)h->b32;
    v.n = h->n_active;
    v.ilu = IluView<T32>{};
    if (has_ilu(h)) {
        v.ilu.rp = h->ilu_rp;
        v.ilu.ci = h->ilu_ci;
        v.ilu.lu = (const T32 *)h->ilu_lu32;
        v.ilu.dpos = h->ilu_dpos;
        v.ilu.lrows = h->ilu_lrows;
        v.ilu.lptr = h->ilu_lptr;
        v.ilu.urows = h->ilu_urows;
        v.ilu.uptr = h->ilu_uptr;
        v.ilu.nlev_l = h->ilu_nlev_l;
        v.ilu.nlev_u = h->ilu_nlev_u;
        v.ilu.nnz = h->ilu_nnz;
        v.ilu.t = (T32 *)h->ilu_t32;
        v.ilu.lcnt = h->ilu_lcnt;
        v.ilu.ucnt = h->ilu_ucnt;
        v.ilu.lell_c = h->ilu_lell_c;
        v.ilu.uell_c = h->ilu_uell_c;
        v.ilu.lell_a = (const T32 *)h->ilu_lell_a32;
        v.ilu.uell_a = (const T32 *)h->ilu_uell_a32;
        v.ilu.udiag = (const T32 *)h->ilu_udiag32;
    }
    return v;
}

template <typename T64>
RefView<T64> make_ref_view(const mlb_handle *h) {
    RefView<T64> v;
    v.N = h->N;
    v.ld = h->ld;
    v.nnz = h->nnz;
    v.nslices = h->nslices;
    v.slice_ptr = h->slice_ptr;
    v.scol = h->scol;
    v.sval = (const T64 *)h->sval;
    set_spt(v.spt, h->maxw, sizeof(T64), h->spt_cap, h->ew);
    v.x = (T64 *)h->x;
    v.b = (const T64 *)h->b;
    v.r = (T64 *)h->r;
    v.xbest = (T64 *)h->xbest;
    return v;
}

// Controls of the refined mode's inner calls: reliable-update factor,
// iteration cap, stagnation window (iterations without a new smallest
// residual at a block end).
constexpr int64_t kStallWindow = 2000;
RefCtl ref_ctl(const mlb_handle *h) {
    RefCtl rc;
    rc.delta = h->inner_tol;
    rc.inner_maxit = h->inner_maxit;
    rc.window = kStallWindow;
    return rc;
}

// Device memory of GPU `dev` (the handle's), or managed memory.  Memory of
// another GPU is refused: the kernels run on `dev`.
bool is_device_ptr(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Inputs of a solve into the handle's b and x (the caller's row order, or
// the multicolour order: b_B = P b, x_B = P x), and the solution back.
int stage_in(mlb_handle *h, const void *b, const void *x, int32_t on_device, cudaStream_t st) {
    const size_t nb = (size_t)h->N * h->esize;
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (h->perm_h.empty()) {
        MLB_CUDA(cudaMemcpyAsync(h->b, b, nb, in, st));
        MLB_CUDA(cudaMemcpyAsync(h->x, x, nb, in, st));
        return MLB_OK;
    }
    MLB_CUDA(cudaMemcpyAsync(h->pstage, b, nb, in, st));
    MLB_CUDA(launch_permute(h->pstage, h->b, h->perm_d, h->N, (int)h->esize, true, st));
    MLB_CUDA(cudaMemcpyAsync(h->pstage, x, nb, in, st));
    MLB_CUDA(launch_permute(h->pstage, h->x, h->perm_d, h->N, (int)h->esize, true, st));
    return MLB_OK;
}
int stage_out(mlb_handle *h, void *x, int32_t on_device, cudaStream_t st) {
    const size_t nb = (size_t)h->N * h->esize;
    const cudaMemcpyKind outk = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (h->perm_h.empty()) {
        MLB_CUDA(cudaMemcpyAsync(x, h->x, nb, outk, st));
        return MLB_OK;
    }
    MLB_CUDA(launch_permute(h->x, h->pstage, h->perm_d, h->N, (int)h->esize, false, st));
    MLB_CUDA(cudaMemcpyAsync(x, h->pstage, nb, outk, st));
    return MLB_OK;
}

// With a preconditioner the kernels iterate on y = M x (A M^{-1} y = b):
// before a solve the caller's x_0 becomes y_0 = M x_0, afterwards the
// result y becomes x = M^{-1} y, on the handle's buffer h->x.  Here for
// the Jacobi M; the solve kernel maps ILU(0) itself.
int map_solution(mlb_handle *h, bool to_x, cudaStream_t st) {
    if (h->precond != MLB_PRECOND_JACOBI) return MLB_OK;
    cudaError_t e = h->dtype == MLB_C128
                        ? launch_diag_apply<cdouble>((cdouble *)h->x, (const cdouble *)h->mdiag, h->N, to_x, st)
                        : launch_diag_apply<double>((double *)h->x, (const double *)h->mdiag, h->N, to_x, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    return MLB_OK;
}
int map_solution(mlb_handle *h, bool to_x) { return map_solution(h, to_x, h->stream); }

static_assert(Engine<double, true>::kIluReg == kIluEll, "ILU(0) entries held by position = entries in registers");

// Jacobi preconditioner M = diag(A) (Algorithm 7.1, right preconditioning):
// d = diagonal of A (a row's diagonal entries summed), values of A M^{-1}
// (column j divided by d_j) and, when A^H is supplied, of M^{-H} A^H (row i
// divided by conj(d_i)).  MLB_ERR_ARG when some d_i is zero or not finite.
template <typename V>
int jacobi_scale_t(const mlb_matrix *A, const mlb_matrix *AH, std::vector<char> &dg, std::vector<char> &av,
                   std::vector<char> &ahv) {
    const int64_t N = A->nrows;
    std::vector<V> d(N, V(0));
    const V *a = (const V *)A->values;
    for (int64_t r = 0; r < N; ++r)
        for (int64_t k = A->row_ptr[r]; k < A->row_ptr[r + 1]; ++k)
            if (A->col_idx[k] == r) d[r] += a[k];
    for (int64_t r = 0; r < N; ++r)
        if (!(std::abs(d[r]) > 0.0) || !std::isfinite(std::abs(d[r]))) return MLB_ERR_ARG;
    dg.assign((const char *)d.data(), (const char *)(d.data() + N));
    av.resize((size_t)A->nnz * sizeof(V));
    V *o = (V *)av.data();
    for (int64_t k = 0; k < A->nnz; ++k) o[k] = a[k] / d[A->col_idx[k]];
    if (AH) {
        ahv.resize((size_t)AH->nnz * sizeof(V));
        const V *ah = (const V *)AH->values;
        V *oh = (V *)ahv.data();
        for (int64_t r = 0; r < N; ++r)
            for (int64_t k = AH->row_ptr[r]; k < AH->row_ptr[r + 1]; ++k) {
                if constexpr (std::is_same<V, double>::value) oh[k] = ah[k] / d[r];
                else oh[k] = ah[k] / std::conj(d[r]);
            }
    }
    return MLB_OK;
}

int create_impl(mlb_handle *h, const mlb_matrix *A, const mlb_matrix *AH, const mlb_options *o) {
    MLB_CUDA(cudaGetDevice(&h->device));
    h->dtype = A->dtype;
    h->esize = A->dtype == MLB_C128 ? 16 : 8;
    h->n = o->n;
    h->n_active = o->n;
    h->precond = o->precond;
    // BSR(3) input: the host-side steps (factors, orderings, A^H) work on
    // the scalar CSR; the products keep one column per block row segment
    std::vector<int64_t> xrp, xhrp;
    std::vector<int32_t> xci, xhci;
    std::vector<char> xval, xhval;
    mlb_matrix Xm, XHm;
    if (A->block == 3) {
        bsr3_expand(A, h->esize, xrp, xci, xval);
        Xm = *A;
        Xm.block = 1;
        Xm.nnz = xrp.back();
        Xm.row_ptr = xrp.data();
        Xm.col_idx = xci.data();
        Xm.values = xval.data();
        A = &Xm;
    }
    if (AH && AH->block == 3) {
        bsr3_expand(AH, h->esize, xhrp, xhci, xhval);
        XHm = *AH;
        XHm.block = 1;
        XHm.nnz = xhrp.back();
        XHm.row_ptr = xhrp.data();
        XHm.col_idx = xhci.data();
        XHm.values = xhval.data();
        AH = &XHm;
    }
    // multicolour ILU(0): the handle holds B = P A P^T (and B^H = P A^H P^T),
    // solves B y = P b and returns x = P^T y
    std::vector<int64_t> brp, bhrp;
    std::vector<int32_t> bci, bhci, iperm;
    std::vector<char> bval, bhval;
    mlb_matrix Bm, BHm;
    if (o->precond == MLB_PRECOND_ILU0_MC) {
        h->ncolors = mc_order(A, h->perm_h);
        iperm.assign(A->nrows, 0);
        for (int64_t r = 0; r < A->nrows; ++r) iperm[h->perm_h[r]] = (int32_t)r;
        permute_csr(A, h->perm_h, iperm, h->esize, brp, bci, bval);
        Bm = *A;
        Bm.row_ptr = brp.data();
        Bm.col_idx = bci.data();
        Bm.values = bval.data();
        A = &Bm;
        if (AH) {
            permute_csr(AH, h->perm_h, iperm, h->esize, bhrp, bhci, bhval);
            BHm = *AH;
            BHm.row_ptr = bhrp.data();
            BHm.col_idx = bhci.data();
            BHm.values = bhval.data();
            AH = &BHm;
        }
    }
    // ILU(0): factors and level sets on the host (the handle keeps A itself)
    IluHost ih;
    if (has_ilu(h)) {
        const int rci = ilu0_build(A, ih);
        if (rci) return rci;
    }
    // with a Jacobi preconditioner the handle stores A M^{-1} (and M^{-H} A^H)
    std::vector<char> jd, jav, jahv;
    mlb_matrix As, AHs;
    if (o->precond == MLB_PRECOND_JACOBI) {
        const int rcj = A->dtype == MLB_C128 ? jacobi_scale_t<std::complex<double>>(A, AH, jd, jav, jahv)
                                             : jacobi_scale_t<double>(A, AH, jd, jav, jahv);
        if (rcj) return rcj;
        As = *A;
        As.values = jav.data();
        A = &As;
        if (AH) {
            AHs = *AH;
            AHs.values = jahv.data();
            AH = &AHs;
        }
    }
    h->precision = o->precision;
    h->N = A->nrows;
    h->nnz = A->nnz;
    h->ld = round_up(h->N, 512);
    h->nslices = h->ld / 32;
    h->stream = (cudaStream_t)o->stream;
    h->timeout_ns = (uint64_t)o->timeout_ns;
    h->kappa = o->kappa;
    h->max_outer = o->max_outer;
    h->inner_tol = o->inner_tol;
    h->inner_maxit = o->inner_maxit;
    const size_t es = h->esize;
    const bool cplx = A->dtype == MLB_C128;
    const int64_t ld = h->ld;
    const int n = h->n;
    cudaStream_t st = h->stream;

    // matrix in SELL-32
    {
        std::vector<int64_t> sp;
        std::vector<int32_t> col;
        std::vector<char> val;
        h->ew = (!cplx && has_triplets(A)) ? 3 : 1;
        h->maxw = csr_to_sell32(A, ld, sp, col, val, es, h->ew);
        h->nnz_pad = sp.back();
        int rc;
        if ((rc = dev_alloc_t(h, &h->slice_ptr, sp.size() * 8))) return rc;
        if ((rc = dev_alloc_t(h, &h->scol, col.size() * 4))) return rc;
        if ((rc = dev_alloc(h, &h->sval, val.size()))) return rc;
        MLB_CUDA(cudaMemcpy(h->slice_ptr, sp.data(), sp.size() * 8, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->scol, col.data(), col.size() * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->sval, val.data(), val.size(), cudaMemcpyHostToDevice));
    }
    // vectors: Q, F, G, W (ld x n), x, r, z, b (ld), zero padded
    int rc;
    const size_t vb = (size_t)ld * es;
    if ((rc = dev_alloc(h, &h->Q, vb * n))) return rc;
    if (n > 1 && (rc = dev_alloc(h, &h->F, vb * (n - 1)))) return rc;
    const bool refined = h->precision == MLB_PREC_FP32_REFINED;
    if (!refined) {
        if ((rc = dev_alloc(h, &h->G, vb * n))) return rc;
        if ((rc = dev_alloc(h, &h->W, vb * n))) return rc;
        if ((rc = dev_alloc(h, &h->z, vb))) return rc;
        MLB_CUDA(cudaMemsetAsync(h->G, 0, vb * n, st));
        MLB_CUDA(cudaMemsetAsync(h->W, 0, vb * n, st));
        MLB_CUDA(cudaMemsetAsync(h->z, 0, vb, st));
    }
    if ((rc = dev_alloc(h, &h->x, vb))) return rc;
    if ((rc = dev_alloc(h, &h->r, vb))) return rc;
    if ((rc = dev_alloc(h, &h->b, vb))) return rc;
    MLB_CUDA(cudaMemsetAsync(h->Q, 0, vb * n, st));
    if (n > 1) MLB_CUDA(cudaMemsetAsync(h->F, 0, vb * (n - 1), st));
    MLB_CUDA(cudaMemsetAsync(h->x, 0, vb, st));
    MLB_CUDA(cudaMemsetAsync(h->r, 0, vb, st));
    MLB_CUDA(cudaMemsetAsync(h->b, 0, vb, st));
    if (h->precond == MLB_PRECOND_JACOBI) {
        if ((rc = dev_alloc(h, &h->mdiag, vb))) return rc;
        MLB_CUDA(cudaMemcpy(h->mdiag, jd.data(), (size_t)h->N * es, cudaMemcpyHostToDevice));
    }
    if (has_ilu(h)) {
        const int64_t N = h->N;
        h->ilu_nnz = ih.nnz;
        h->ilu_nlev_l = ih.nlev_l;
        h->ilu_nlev_u = ih.nlev_u;
        if ((rc = dev_alloc_t(h, &h->ilu_rp, (size_t)(N + 1) * 8))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_ci, (size_t)ih.nnz * 4))) return rc;
        if ((rc = dev_alloc(h, &h->ilu_lu, (size_t)ih.nnz * es))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_dpos, (size_t)N * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_lrows, (size_t)N * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_lptr, ih.lptr.size() * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_urows, (size_t)N * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_uptr, ih.uptr.size() * 4))) return rc;
        if ((rc = dev_alloc(h, &h->ilu_t, vb))) return rc;
        MLB_CUDA(cudaMemcpy(h->ilu_rp, ih.rp.data(), (size_t)(N + 1) * 8, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_ci, ih.ci.data(), (size_t)ih.nnz * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_lu, ih.lu.data(), (size_t)ih.nnz * es, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_dpos, ih.dpos.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_lrows, ih.lrows.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_lptr, ih.lptr.data(), ih.lptr.size() * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_urows, ih.urows.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_uptr, ih.uptr.data(), ih.uptr.size() * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemsetAsync(h->ilu_t, 0, vb, st));
        const size_t ne = (size_t)kIluEll * N;
        if ((rc = dev_alloc_t(h, &h->ilu_lcnt, (size_t)N * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_ucnt, (size_t)N * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_lell_c, ne * 4))) return rc;
        if ((rc = dev_alloc_t(h, &h->ilu_uell_c, ne * 4))) return rc;
        if ((rc = dev_alloc(h, &h->ilu_lell_a, ne * es))) return rc;
        if ((rc = dev_alloc(h, &h->ilu_uell_a, ne * es))) return rc;
        if ((rc = dev_alloc(h, &h->ilu_udiag, (size_t)N * es))) return rc;
        MLB_CUDA(cudaMemcpy(h->ilu_lcnt, ih.lcnt.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_ucnt, ih.ucnt.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_lell_c, ih.lell_c.data(), ne * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_uell_c, ih.uell_c.data(), ne * 4, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_lell_a, ih.lell_a.data(), ne * es, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_uell_a, ih.uell_a.data(), ne * es, cudaMemcpyHostToDevice));
        MLB_CUDA(cudaMemcpy(h->ilu_udiag, ih.udiag.data(), (size_t)N * es, cudaMemcpyHostToDevice));
    }

    // reordering (multicolour ILU(0)): the permutation and a staging vector
    if (!h->perm_h.empty()) {
        if ((rc = dev_alloc_t(h, &h->perm_d, (size_t)h->N * 4))) return rc;
        if ((rc = dev_alloc(h, &h->pstage, vb))) return rc;
        MLB_CUDA(cudaMemcpy(h->perm_d, h->perm_h.data(), (size_t)h->N * 4, cudaMemcpyHostToDevice));
    }
    // shadow vectors (given and drawn in the original row order)
    if (o->Q && !h->perm_h.empty()) {
        std::vector<char> qp((size_t)h->N * n * es);
        const char *qs = (const char *)o->Q;
        for (int m = 0; m < n; ++m)
            for (int64_t r = 0; r < h->N; ++r)
                memcpy(&qp[((size_t)m * h->N + r) * es], qs + ((size_t)m * h->N + h->perm_h[r]) * es, es);
        MLB_CUDA(cudaMemcpy2D(h->Q, ld * es, qp.data(), h->N * es, h->N * es, n, cudaMemcpyHostToDevice));
    } else if (o->Q) {
        MLB_CUDA(cudaMemcpy2DAsync(h->Q, ld * es, o->Q, h->N * es, h->N * es, n, cudaMemcpyHostToDevice, st));
    } else {
        MLB_CUDA(launch_qgen(h->Q, cplx ? 1 : 0, h->N, ld, n, o->q_seed, st, h->perm_d));
    }

    // F = A^H Q(:, 0:n-2) (Algorithm 4.1, step 2)
    if (n > 1) {
        std::vector<int64_t> trp;
        std::vector<int32_t> tci;
        std::vector<char> tav;
        const int64_t *rp;
        const int32_t *ci;
        const void *av;
        int64_t tnnz;
        if (AH) {
            rp = AH->row_ptr;
            ci = AH->col_idx;
            av = AH->values;
            tnnz = AH->nnz;
        } else {
            conj_transpose(A, trp, tci, tav, es, cplx);
            rp = trp.data();
            ci = tci.data();
            av = tav.data();
            tnnz = A->nnz;
        }
        int64_t *drp = nullptr;
        int32_t *dci = nullptr;
        void *dav = nullptr;
        if (cudaMalloc(&drp, (h->N + 1) * 8) != cudaSuccess ||
            cudaMalloc(&dci, std::max<int64_t>(tnnz, 1) * 4) != cudaSuccess ||
            cudaMalloc(&dav, std::max<int64_t>(tnnz, 1) * es) != cudaSuccess) {
            cudaFree(drp);
            cudaFree(dci);
            cudaFree(dav);
            cudaGetLastError();
            return MLB_ERR_OOM;
        }
        cudaError_t e = cudaMemcpy(drp, rp, (h->N + 1) * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && tnnz) e = cudaMemcpy(dci, ci, tnnz * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && tnnz) e = cudaMemcpy(dav, av, tnnz * es, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            if (cplx)
                e = launch_ahq<cdouble>(drp, dci, (const cdouble *)dav, h->N, ld, (const cdouble *)h->Q,
                                        (cdouble *)h->F, n - 1, st);
            else
                e = launch_ahq<double>(drp, dci, (const double *)dav, h->N, ld, (const double *)h->Q,
                                       (double *)h->F, n - 1, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(drp);
        cudaFree(dci);
        cudaFree(dav);
        if (e != cudaSuccess) return MLB_ERR_CUDA;
        // ILU(0): F = M^{-H} (A^H Q), column by column on the host
        if (has_ilu(h)) {
            std::vector<char> col((size_t)h->N * es);
            for (int m = 0; m < n - 1; ++m) {
                char *dcol = (char *)h->F + (size_t)m * ld * es;
                MLB_CUDA(cudaMemcpy(col.data(), dcol, col.size(), cudaMemcpyDeviceToHost));
                ilu0_apply_h(ih, cplx, col.data());
                MLB_CUDA(cudaMemcpy(dcol, col.data(), col.size(), cudaMemcpyHostToDevice));
            }
        }
    }

    // refined mode: FP32 copies of the values, Q and F; FP32 work vectors
    if (refined) {
        const size_t vb32 = vb / 2;
        if ((rc = dev_alloc(h, &h->sval32, (size_t)h->nnz_pad * h->ew * es / 2))) return rc;
        if ((rc = dev_alloc(h, &h->Q32, vb32 * n))) return rc;
        if (n > 1 && (rc = dev_alloc(h, &h->F32, vb32 * (n - 1)))) return rc;
        if ((rc = dev_alloc(h, &h->G32, vb32 * n))) return rc;
        if ((rc = dev_alloc(h, &h->W32, vb32 * n))) return rc;
        if ((rc = dev_alloc(h, &h->x32, vb32))) return rc;
        if ((rc = dev_alloc(h, &h->r32, vb32))) return rc;
        if ((rc = dev_alloc(h, &h->z32, vb32))) return rc;
        if ((rc = dev_alloc(h, &h->b32, vb32))) return rc;
        if ((rc = dev_alloc(h, &h->xbest, vb))) return rc;
        MLB_CUDA(cudaMemsetAsync(h->xbest, 0, vb, st));
        MLB_CUDA(cudaMemsetAsync(h->G32, 0, vb32 * n, st));
        MLB_CUDA(cudaMemsetAsync(h->W32, 0, vb32 * n, st));
        MLB_CUDA(cudaMemsetAsync(h->x32, 0, vb32, st));
        MLB_CUDA(cudaMemsetAsync(h->r32, 0, vb32, st));
        MLB_CUDA(cudaMemsetAsync(h->z32, 0, vb32, st));
        MLB_CUDA(cudaMemsetAsync(h->b32, 0, vb32, st));
        MLB_CUDA(launch_narrow((const double *)h->sval, (float *)h->sval32, h->nnz_pad * h->ew * (int64_t)es / 8, st));
        MLB_CUDA(launch_narrow((const double *)h->Q, (float *)h->Q32, ld * (int64_t)n * (int64_t)es / 8, st));
        if (n > 1)
            MLB_CUDA(launch_narrow((const double *)h->F, (float *)h->F32, ld * (int64_t)(n - 1) * (int64_t)es / 8,
                                   st));
        if (has_ilu(h)) {
            const int64_t N = h->N;
            const size_t ne = (size_t)kIluEll * N;
            if ((rc = dev_alloc(h, &h->ilu_lu32, (size_t)h->ilu_nnz * es / 2))) return rc;
            if ((rc = dev_alloc(h, &h->ilu_t32, vb32))) return rc;
            if ((rc = dev_alloc(h, &h->ilu_lell_a32, ne * es / 2))) return rc;
            if ((rc = dev_alloc(h, &h->ilu_uell_a32, ne * es / 2))) return rc;
            if ((rc = dev_alloc(h, &h->ilu_udiag32, (size_t)N * es / 2))) return rc;
            MLB_CUDA(cudaMemsetAsync(h->ilu_t32, 0, vb32, st));
            const int64_t dpe = (int64_t)es / 8;   // doubles per value
            MLB_CUDA(launch_narrow((const double *)h->ilu_lu, (float *)h->ilu_lu32, h->ilu_nnz * dpe, st));
            MLB_CUDA(launch_narrow((const double *)h->ilu_lell_a, (float *)h->ilu_lell_a32, (int64_t)ne * dpe, st));
            MLB_CUDA(launch_narrow((const double *)h->ilu_uell_a, (float *)h->ilu_uell_a32, (int64_t)ne * dpe, st));
            MLB_CUDA(launch_narrow((const double *)h->ilu_udiag, (float *)h->ilu_udiag32, N * dpe, st));
        }
    }

    // launch geometry and scratch
    int sms = 0;
    MLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int bps = refined ? (cplx ? refine_blocks_per_sm<cfloat, cdouble>() : refine_blocks_per_sm<float, double>())
                            : (cplx ? solve_blocks_per_sm<cdouble>() : solve_blocks_per_sm<double>());
    if (bps < 1) return MLB_ERR_CUDA;
    const int64_t nchunk = ld * (int64_t)es / 16;
    int64_t want = (nchunk + kThreads - 1) / kThreads;
    int maxg = sms * bps;
    int grid = (int)std::min<int64_t>(want, maxg);
    if (o->grid > 0) grid = std::min(o->grid, maxg);
    h->grid = std::max(grid, 1);
    h->grid_max = std::max(maxg, 1);
    h->grid_want = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxg));
    if ((rc = dev_alloc_t(h, &h->partials, (size_t)2 * maxg * kMaxSums * 8))) return rc;
    if ((rc = dev_alloc_t(h, &h->bar, sizeof(BarrierState)))) return rc;
    if ((rc = dev_alloc_t(h, &h->dres, sizeof(DevResult)))) return rc;
    if ((rc = dev_alloc_t(h, &h->qd_partials, (size_t)h->grid_max * kQdMaxN * 2 * 8))) return rc;
    if ((rc = dev_alloc_t(h, &h->qd_out, (size_t)(kQdMaxN * 2 + 1) * 8))) return rc;
    if ((rc = dev_alloc_t(h, &h->qd_status, (size_t)h->grid_max * sizeof(int)))) return rc;
    if ((rc = dev_alloc_t(h, &h->qd_ticket, sizeof(unsigned)))) return rc;
    MLB_CUDA(cudaMemsetAsync(h->qd_ticket, 0, sizeof(unsigned), st));
    if (cudaMallocHost(&h->qd_host, (size_t)(kQdMaxN * 2 + 1) * 8) != cudaSuccess) {
        cudaGetLastError();
        h->qd_host = nullptr;
        return MLB_ERR_OOM;
    }
    if (cudaMallocHost(&h->hres, sizeof(DevResult)) != cudaSuccess) {
        cudaGetLastError();
        h->hres = nullptr;
        return MLB_ERR_OOM;
    }
    MLB_CUDA(cudaEventCreate(&h->ev0));
    MLB_CUDA(cudaEventCreate(&h->ev1));
    MLB_CUDA(cudaStreamSynchronize(st));
    return MLB_OK;
}

void release(mlb_handle *h) {
    if (!h) return;
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->err_hist) cudaFree(h->err_hist);
    if (h->hres) cudaFreeHost(h->hres);
    if (h->qd_host) cudaFreeHost(h->qd_host);
    if (h->bws) cudaFree(h->bws);
    if (h->bhost) cudaFreeHost(h->bhost);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaGetLastError();
}

}  // namespace

extern "C" {

void mlbicgstab_default_options(mlb_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->n = 4;
    o->precision = MLB_PREC_FP64;
    o->q_seed = 0;
    o->Q = nullptr;
    o->kappa = 0.0;
    o->max_outer = 10;
    o->grid = 0;
    o->inner_tol = 1e-2;
    o->inner_maxit = 1000000;
    o->stream = nullptr;
    o->timeout_ns = 2000000000LL;
}

const char *mlbicgstab_strerror(int code) {
    switch (code) {
        case MLB_OK: return "success";
        case MLB_ERR_ARG: return "invalid argument";
        case MLB_ERR_CUDA: return "CUDA runtime error or no CUDA device";
        case MLB_ERR_OOM: return "out of memory";
        case MLB_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case MLB_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status code";
    }
}

int mlbicgstab_create(mlb_handle **out, const mlb_matrix *A, const mlb_matrix *AH, const mlb_options *opt) {
    if (!out) return MLB_ERR_ARG;
    *out = nullptr;
    mlb_options o;
    if (opt) o = *opt;
    else mlbicgstab_default_options(&o);
    if (o.n < 1 || o.n > kMaxN) return MLB_ERR_ARG;
    if (o.precision != MLB_PREC_FP64 && o.precision != MLB_PREC_FP32_REFINED) return MLB_ERR_ARG;
    if (o.kappa < 0.0 || o.max_outer < 0 || o.timeout_ns <= 0) return MLB_ERR_ARG;
    if (o.precision == MLB_PREC_FP32_REFINED && (!(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.inner_maxit < 1))
        return MLB_ERR_ARG;
    if ((o.precond != MLB_PRECOND_NONE && o.precond != MLB_PRECOND_JACOBI && o.precond != MLB_PRECOND_ILU0 &&
         o.precond != MLB_PRECOND_ILU0_MC) ||
        o.reserved0 != 0)
        return MLB_ERR_ARG;
    int rc = validate_csr(A);
    if (rc) return rc;
    if (AH) {
        rc = validate_csr(AH);
        if (rc) return rc;
        if (AH->nrows != A->nrows || AH->dtype != A->dtype) return MLB_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    mlb_handle *h = new (std::nothrow) mlb_handle();
    if (!h) return MLB_ERR_OOM;
    rc = create_impl(h, A, AH, &o);
    if (rc) {
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return MLB_OK;
}

void mlbicgstab_destroy(mlb_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

int mlbicgstab_info(const mlb_handle *h, mlb_info *info) {
    if (!h || !info) return MLB_ERR_ARG;
    memset(info, 0, sizeof(*info));
    info->nrows = h->N;
    info->nnz = h->nnz;
    info->n = h->n;
    info->n_active = h->n_active;
    info->precond = h->precond;
    info->entry_values = h->ew;
    info->ilu_levels = has_ilu(h) ? h->ilu_nlev_l : 0;
    info->dtype = h->dtype;
    info->precision = h->precision;
    info->grid = h->grid;
    info->block = kThreads;
    info->nnz_padded = h->nnz_pad;
    info->device_bytes = h->device_bytes;
    info->qd_kernel_ms = h->qd_ms;
    return MLB_OK;
}

int mlbicgstab_get_Q(const mlb_handle *h, void *host_out) {
    if (!h || !host_out) return MLB_ERR_ARG;
    MLB_CUDA(cudaSetDevice(h->device));
    MLB_CUDA(cudaMemcpy2DAsync(host_out, h->N * h->esize, h->Q, h->ld * h->esize, h->N * h->esize, h->n,
                               cudaMemcpyDeviceToHost, h->stream));
    MLB_CUDA(cudaStreamSynchronize(h->stream));
    if (!h->perm_h.empty()) {   // back to the original row order
        const size_t es = h->esize;
        std::vector<char> tmp((size_t)h->N * es);
        char *q = (char *)host_out;
        for (int m = 0; m < h->n; ++m) {
            char *col = q + (size_t)m * h->N * es;
            memcpy(tmp.data(), col, tmp.size());
            for (int64_t r = 0; r < h->N; ++r) memcpy(col + (size_t)h->perm_h[r] * es, &tmp[(size_t)r * es], es);
        }
    }
    return MLB_OK;
}

int mlbicgstab_get_perm(const mlb_handle *h, int32_t *host_out) {
    if (!h || !host_out) return MLB_ERR_ARG;
    for (int64_t r = 0; r < h->N; ++r) host_out[r] = h->perm_h.empty() ? (int32_t)r : h->perm_h[r];
    return MLB_OK;
}

int mlbicgstab_solve(mlb_handle *h, const void *b, void *x, int32_t on_device, double tol, int64_t maxit,
                     mlb_result *res, double *err_hist, int64_t hist_cap) {
    if (!h || !b || !x || !res) return MLB_ERR_ARG;
    if (!(tol >= 0.0) || maxit < 0 || hist_cap < 0 || (on_device != 0 && on_device != 1)) return MLB_ERR_ARG;
    memset(res, 0, sizeof(*res));
    MLB_CUDA(cudaSetDevice(h->device));
    if (on_device && (!is_device_ptr(b, h->device) || !is_device_ptr(x, h->device))) return MLB_ERR_ARG;
    cudaStream_t st = h->stream;
    if (err_hist && hist_cap > h->err_cap) {
        if (h->err_hist) cudaFree(h->err_hist);
        h->err_hist = nullptr;
        h->err_cap = 0;
        if (cudaMalloc(&h->err_hist, hist_cap * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return MLB_ERR_OOM;
        }
        h->err_cap = hist_cap;
    }
    if (int rcs = stage_in(h, b, x, on_device, st)) return rcs;
    if (int rcm = map_solution(h, false)) return rcm;   // y_0 = M x_0
    MLB_CUDA(cudaMemsetAsync(h->bar, 0, sizeof(BarrierState), st));
    SolveCtl ctl;
    ctl.tol = tol;
    ctl.maxit = maxit;
    ctl.kappa = h->kappa;
    ctl.max_outer = h->max_outer;
    ctl.err_hist = err_hist ? h->err_hist : nullptr;
    ctl.hist_cap = err_hist ? hist_cap : 0;
    ctl.partials = h->partials;
    ctl.bar = h->bar;
    ctl.res = h->dres;
    ctl.timeout_ns = h->timeout_ns;
    MLB_CUDA(cudaEventRecord(h->ev0, st));
    cudaError_t e;
    if (h->precision == MLB_PREC_FP32_REFINED) {
        const RefCtl rc = ref_ctl(h);
        if (h->dtype == MLB_C128)
            e = launch_refine<cfloat, cdouble>(make_view32<cfloat>(h), make_ref_view<cdouble>(h), ctl, rc, h->grid,
                                               st);
        else
            e = launch_refine<float, double>(make_view32<float>(h), make_ref_view<double>(h), ctl, rc, h->grid, st);
    } else if (h->dtype == MLB_C128) {
        e = launch_solve<cdouble>(make_view<cdouble>(h), ctl, h->grid, st);
    } else {
        e = launch_solve<double>(make_view<double>(h), ctl, h->grid, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    MLB_CUDA(cudaEventRecord(h->ev1, st));
    if (int rcm = map_solution(h, true)) return rcm;    // x = M^{-1} y
    if (int rcs = stage_out(h, x, on_device, st)) return rcs;
    MLB_CUDA(cudaMemcpyAsync(h->hres, h->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, st));
    MLB_CUDA(cudaStreamSynchronize(st));
    const DevResult &d = *h->hres;
    res->flag = d.flag;
    res->j = d.j;
    res->i = d.i;
    res->status = d.status;
    res->iter = d.iter;
    res->spmv = d.spmv;
    res->outer = d.outer;
    res->err = d.err;
    res->true_relres = d.true_relres;
    res->bytes = d.bytes;
    res->flops = d.flops;
    for (int q = 0; q < 5; ++q) res->ops[q] = d.ops[q];
    res->ctas = d.ctas;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    res->kernel_ms = ms;
    if (err_hist && hist_cap > 0) {
        int64_t cnt = std::min<int64_t>(hist_cap, d.iter + 1);
        for (int64_t k = 0; k < hist_cap; ++k) err_hist[k] = __builtin_nan("");
        if (cnt > 0) MLB_CUDA(cudaMemcpy(err_hist, h->err_hist, cnt * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (d.status != 0) return MLB_ERR_TIMEOUT;
    return MLB_OK;
}

int mlbicgstab_batch_plan(const int64_t *N, const int64_t *nnz, const int32_t *precond, int32_t count,
                          int32_t team, int32_t slots, int32_t *ctas, int32_t *order, int32_t *nbig,
                          int32_t *teams, int32_t *grid) {
    if (!N || !nnz || !precond || count <= 0 || team < 1 || slots < 1 || !ctas || !order || !nbig || !teams ||
        !grid)
        return MLB_ERR_ARG;
    for (int32_t s = 0; s < count; ++s)
        if (N[s] < 1 || nnz[s] < 0) return MLB_ERR_ARG;
    // Estimated work w = (nnz + N) N^(1/3); systems of at least
    // kTeamMinRows rows per team CTA whose w exceeds kTeamShare of the
    // average per CTA go to teams, the others to single CTAs; each list
    // largest first (longest-processing-time order).  Natural-order ILU(0)
    // systems stay on one CTA: their triangular solves take one barrier
    // per level, which a team pays in global memory (measured: the 512-
    // system ILU(0) batch 2.20 s with teams of 4, 1.96 s without).
    const int tm = std::max(1, std::min(team, slots));
    std::vector<double> w(count);
    double wsum = 0.0;
    for (int s = 0; s < count; ++s) {
        w[s] = (double)(nnz[s] + N[s]) * std::cbrt((double)N[s]);
        wsum += w[s];
    }
    std::vector<int> big, small;
    for (int s = 0; s < count; ++s) {
        const bool t = tm > 1 && precond[s] != MLB_PRECOND_ILU0 && N[s] >= (int64_t)kTeamMinRows * tm &&
                       w[s] > kTeamShare * wsum / slots;
        (t ? big : small).push_back(s);
        ctas[s] = t ? tm : 1;
    }
    auto by_work = [&](int a, int c) { return w[a] > w[c]; };
    std::stable_sort(big.begin(), big.end(), by_work);
    std::stable_sort(small.begin(), small.end(), by_work);
    int k = 0;
    for (int s : big) order[k++] = s;
    for (int s : small) order[k++] = s;
    *nbig = (int32_t)big.size();
    *teams = std::min<int>((int)big.size(), slots / tm);
    *grid = std::min(slots, *teams * tm + (int)small.size());
    return MLB_OK;
}

int mlbicgstab_solve_batch(mlb_handle *const *hs, int32_t count, const void *const *b, void *const *x,
                           int32_t on_device, const double *tol, const int64_t *maxit, mlb_result *res) {
    if (!hs || count <= 0 || !b || !x || !tol || !maxit || !res) return MLB_ERR_ARG;
    if (on_device != 0 && on_device != 1) return MLB_ERR_ARG;
    mlb_handle *h0 = hs[0];
    if (!h0) return MLB_ERR_ARG;
    for (int32_t s = 0; s < count; ++s) {
        const mlb_handle *h = hs[s];
        if (!h || !b[s] || !x[s] || !(tol[s] >= 0.0) || maxit[s] < 0) return MLB_ERR_ARG;
        if (h->dtype != h0->dtype || h->precision != h0->precision || h->device != h0->device)
            return MLB_ERR_ARG;
        if (h->ew != 1) return MLB_ERR_UNSUPPORTED;   // the batch kernels take scalar storage
    }
    memset(res, 0, sizeof(mlb_result) * (size_t)count);
    MLB_CUDA(cudaSetDevice(h0->device));
    cudaStream_t st = h0->stream;
    const bool refined = h0->precision == MLB_PREC_FP32_REFINED;
    const bool cplx = h0->dtype == MLB_C128;
    const size_t item_bytes = refined ? (cplx ? sizeof(BatchItemR<cfloat, cdouble>) : sizeof(BatchItemR<float, double>))
                                      : (cplx ? sizeof(BatchItem<cdouble>) : sizeof(BatchItem<double>));
    int sms = 0;
    MLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h0->device));
    const int bps = refined ? (cplx ? batch_refine_blocks_per_sm<cfloat, cdouble>()
                                    : batch_refine_blocks_per_sm<float, double>())
                            : (cplx ? batch_blocks_per_sm<cdouble>() : batch_blocks_per_sm<double>());
    if (bps < 1) return MLB_ERR_CUDA;
    const int slots = sms * bps;   // co-resident CTAs
    std::vector<int64_t> pn(count), pz(count);
    std::vector<int32_t> pp(count), pctas(count), porder(count);
    for (int s = 0; s < count; ++s) {
        pn[s] = hs[s]->N;
        pz[s] = hs[s]->nnz;
        pp[s] = hs[s]->precond;
    }
    int32_t teams = 0, grid = 0, nbig = 0;
    if (int rcp = mlbicgstab_batch_plan(pn.data(), pz.data(), pp.data(), count, h0->batch_team, slots, pctas.data(),
                                        porder.data(), &nbig, &teams, &grid))
        return rcp;
    const int team = std::max(1, std::min(h0->batch_team, slots));
    const std::vector<int> big(porder.begin(), porder.begin() + nbig), small(porder.begin() + nbig, porder.end());
    // workspace: [queue (256 B)] [order_big] [order_small] [team barriers]
    // [team slots] [solve barriers] [results] (copied from the host:
    // zeroes, results marked as not run) [items] [team partial sums]
    auto up256 = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t off_big = 256;
    const size_t off_small = off_big + up256(big.size() * 4 + 4);
    const size_t off_tbar = off_small + up256(small.size() * 4 + 4);
    const size_t off_titem = off_tbar + up256((size_t)teams * sizeof(BarrierState) + 16);
    const size_t off_sbar = off_titem + up256((size_t)teams * 8 + 8);
    const size_t off_res = off_sbar + up256(big.size() * sizeof(BarrierState) + 16);
    const size_t off_items = off_res + up256((size_t)count * sizeof(DevResult));
    const size_t off_spart = off_items + up256((size_t)count * item_bytes);
    const size_t need = off_spart + big.size() * 2 * kMaxSums * (size_t)team * sizeof(double) + 256;
    if (need > h0->bws_bytes) {
        if (h0->bws) cudaFree(h0->bws);
        h0->bws = nullptr;
        h0->bws_bytes = 0;
        if (cudaMalloc(&h0->bws, need) != cudaSuccess) {
            cudaGetLastError();
            return MLB_ERR_OOM;
        }
        h0->bws_bytes = need;
    }
    if (need > h0->bhost_bytes) {
        if (h0->bhost) cudaFreeHost(h0->bhost);
        h0->bhost = nullptr;
        h0->bhost_bytes = 0;
        if (cudaMallocHost(&h0->bhost, need) != cudaSuccess) {
            cudaGetLastError();
            return MLB_ERR_OOM;
        }
        h0->bhost_bytes = need;
    }
    char *dws = (char *)h0->bws;
    char *hws = (char *)h0->bhost;
    DevResult *dres = (DevResult *)(dws + off_res);
    memset(hws, 0, off_items);
    memcpy(hws + off_big, big.data(), big.size() * 4);
    memcpy(hws + off_small, small.data(), small.size() * 4);
    uint64_t max_timeout = 0;
    for (int s = 0; s < count; ++s) {
        DevResult *r0 = (DevResult *)(hws + off_res) + s;
        r0->flag = 1;
        r0->status = kStatusTimeout;   // a system no CTA took reports a failed wait
        max_timeout = std::max<uint64_t>(max_timeout, hs[s]->timeout_ns);
    }
    for (int s = 0; s < count; ++s) {
        const mlb_handle *h = hs[s];
        SolveCtl ctl;
        memset(&ctl, 0, sizeof(ctl));
        ctl.tol = tol[s];
        ctl.maxit = maxit[s];
        ctl.kappa = h->kappa;
        ctl.max_outer = h->max_outer;
        ctl.res = dres + s;
        ctl.timeout_ns = h->timeout_ns;
        char *dst = hws + off_items + (size_t)s * item_bytes;
        const int cap = batch_cap(h);
        if (refined) {
            const RefCtl rc = ref_ctl(h);
            if (cplx) {
                BatchItemR<cfloat, cdouble> it{make_view32<cfloat>(h), make_ref_view<cdouble>(h), ctl, rc};
                set_spt(it.sys.spt, h->maxw, sizeof(cfloat), cap, h->ew);
                set_spt(it.rv.spt, h->maxw, sizeof(cdouble), cap, h->ew);
                memcpy(dst, &it, sizeof(it));
            } else {
                BatchItemR<float, double> it{make_view32<float>(h), make_ref_view<double>(h), ctl, rc};
                set_spt(it.sys.spt, h->maxw, sizeof(float), cap, h->ew);
                set_spt(it.rv.spt, h->maxw, sizeof(double), cap, h->ew);
                memcpy(dst, &it, sizeof(it));
            }
        } else if (cplx) {
            BatchItem<cdouble> it{make_view<cdouble>(h), ctl};
            set_spt(it.sys.spt, h->maxw, sizeof(cdouble), cap, h->ew);
            memcpy(dst, &it, sizeof(it));
        } else {
            BatchItem<double> it{make_view<double>(h), ctl};
            set_spt(it.sys.spt, h->maxw, sizeof(double), cap, h->ew);
            memcpy(dst, &it, sizeof(it));
        }
    }
    BatchPlan plan;
    plan.order_big = (const int *)(dws + off_big);
    plan.count_big = (int)big.size();
    plan.order_small = (const int *)(dws + off_small);
    plan.count_small = (int)small.size();
    plan.team = team;
    plan.teams = teams;
    plan.queue = (unsigned *)dws;
    plan.tbar = (BarrierState *)(dws + off_tbar);
    plan.team_item = (int *)(dws + off_titem);
    plan.sbar = (BarrierState *)(dws + off_sbar);
    plan.spart = (double *)(dws + off_spart);
    plan.timeout_ns = max_timeout;
    for (int s = 0; s < count; ++s) {
        if (int rcs = stage_in(hs[s], b[s], x[s], on_device, st)) return rcs;
        if (int rcm = map_solution(hs[s], false, st)) return rcm;
    }
    MLB_CUDA(cudaMemcpyAsync(dws, hws, off_spart, cudaMemcpyHostToDevice, st));
    bool any_ilu = false;
    for (int q = 0; q < count; ++q) any_ilu = any_ilu || has_ilu(hs[q]);
    const void *ditems = dws + off_items;
    MLB_CUDA(cudaEventRecord(h0->ev0, st));
    cudaError_t e;
    if (refined) {
        if (cplx)
            e = launch_batch_refine<cfloat, cdouble>((const BatchItemR<cfloat, cdouble> *)ditems, plan, grid, any_ilu,
                                                     st);
        else
            e = launch_batch_refine<float, double>((const BatchItemR<float, double> *)ditems, plan, grid, any_ilu, st);
    } else if (cplx) {
        e = launch_batch<cdouble>((const BatchItem<cdouble> *)ditems, plan, grid, any_ilu, st);
    } else {
        e = launch_batch<double>((const BatchItem<double> *)ditems, plan, grid, any_ilu, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    MLB_CUDA(cudaEventRecord(h0->ev1, st));
    for (int s = 0; s < count; ++s) {
        if (int rcm = map_solution(hs[s], true, st)) return rcm;
        if (int rcs = stage_out(hs[s], x[s], on_device, st)) return rcs;
    }
    DevResult *hres = (DevResult *)(hws + off_res);
    MLB_CUDA(cudaMemcpyAsync(hres, dres, (size_t)count * sizeof(DevResult), cudaMemcpyDeviceToHost, st));
    MLB_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
    int rc = MLB_OK;
    for (int s = 0; s < count; ++s) {
        const DevResult &d = hres[s];
        res[s].flag = d.flag;
        res[s].j = d.j;
        res[s].i = d.i;
        res[s].status = d.status;
        res[s].iter = d.iter;
        res[s].spmv = d.spmv;
        res[s].outer = d.outer;
        res[s].err = d.err;
        res[s].true_relres = d.true_relres;
        res[s].bytes = d.bytes;
        res[s].flops = d.flops;
        res[s].kernel_ms = ms;
        res[s].ctas = d.ctas;
        for (int q = 0; q < 5; ++q) res[s].ops[q] = d.ops[q];
        if (d.status != 0) rc = MLB_ERR_TIMEOUT;
    }
    return rc;
}

}  // extern "C"

namespace {

// Enqueue the fused product on the handle's stream: values of type `vt`
// (the FP64 data, or a refined handle's FP32 copies), d = device array of
// n_active * DS doubles plus the status word.  ev0 is recorded directly
// before the kernel when `timed`.
int qd_enqueue(mlb_handle *h, int32_t vt, const void *x, void *y, double *d, bool timed) {
    const bool narrow = vt == MLB_F32 || vt == MLB_C64;
    const bool cplx = h->dtype == MLB_C128;
    if (vt != (cplx ? MLB_C128 : MLB_F64) && vt != (cplx ? MLB_C64 : MLB_F32)) return MLB_ERR_ARG;
    if (narrow && h->precision != MLB_PREC_FP32_REFINED) return MLB_ERR_UNSUPPORTED;
    cudaStream_t st = h->stream;
    cudaEvent_t ev = timed ? h->ev0 : nullptr;
    // x is gathered from the caller's array (SELL padding columns are
    // clamped below N); y goes to the caller's array and to the handle's
    // padded buffer r, which the inner products stream back
    const int grid = std::max(1, std::min(h->grid_want, h->grid_max));
    // tiles of the product carry the fused columns of Q as epilogue vectors
    const size_t vb = narrow ? h->esize / 2 : h->esize;
    const int ne = qd_ne_for(h, cplx, narrow);
    const int spt = std::min(slices_per_tile(h->maxw, vb, ne), h->spt_cap);
    cudaError_t e;
    if (narrow && cplx)
        e = launch_spmv_qdot_tiled<cfloat>(make_view32<cfloat>(h), ne, h->maxw, spt, (const cfloat *)x, (cfloat *)h->r32,
                                           (cfloat *)y, h->qd_partials, grid, h->qd_status, h->qd_ticket, d, ev,
                                           st);
    else if (narrow)
        e = launch_spmv_qdot_tiled<float>(make_view32<float>(h), ne, h->maxw, spt, (const float *)x, (float *)h->r32,
                                          (float *)y, h->qd_partials, grid, h->qd_status, h->qd_ticket, d, ev, st);
    else if (cplx)
        e = launch_spmv_qdot_tiled<cdouble>(make_view<cdouble>(h), ne, h->maxw, spt, (const cdouble *)x, (cdouble *)h->r,
                                            (cdouble *)y, h->qd_partials, grid, h->qd_status, h->qd_ticket, d, ev,
                                            st);
    else
        e = launch_spmv_qdot_tiled<double>(make_view<double>(h), ne, h->maxw, spt, (const double *)x, (double *)h->r,
                                           (double *)y, h->qd_partials, grid, h->qd_status, h->qd_ticket, d, ev,
                                           st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    return MLB_OK;
}

}  // namespace

extern "C" {

// Autotuner: CTA count and slices per SpMV tile, chosen by timing short
// fixed-length solves on the handle's own matrix, and the columns fused
// into the fused product's epilogue, chosen by timing the product; the
// choice is cached per (dtype, precision, preconditioner, floor(log2 N),
// round(nnz/N), active n).
struct TuneChoice {
    int grid, spt, qd_ne;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int64_t, int>, TuneChoice> g_tune_cache;
// batch autotuner: cap per (dtype, precision, preconditioner, floor(log2 N), round(nnz/N)),
// team size per (dtype, precision, preconditioner, count, floor(log2 of the total N))
static std::map<std::tuple<int, int, int, int, int64_t>, int> g_btune_cache;
static std::map<std::tuple<int, int, int, int, int>, int> g_bteam_cache;

static int log2_floor(int64_t v) {
    int lg = 0;
    for (; v > 1; v >>= 1) ++lg;
    return lg;
}
static int64_t per_row(const mlb_handle *h) {
    return (int64_t)((double)h->nnz / (double)std::max<int64_t>(h->N, 1) + 0.5);
}

// Mean device time of one fused product with `ne` columns fused: 20
// back-to-back launches between two events on the handle's stream, after
// one untimed launch.  x, y: device vectors of N values of type vt; the
// results land in the handle's qd_out, whose status word is checked.
static int time_qd(mlb_handle *h, int32_t vt, int ne, const void *x, void *y, double &us) {
    const int keep = h->qd_ne;
    h->qd_ne = ne;
    cudaStream_t st = h->stream;
    int rc = qd_enqueue(h, vt, x, y, h->qd_out, false);
    if (rc == MLB_OK && cudaEventRecord(h->ev0, st) != cudaSuccess) rc = MLB_ERR_CUDA;
    for (int k = 0; k < 20 && rc == MLB_OK; ++k) rc = qd_enqueue(h, vt, x, y, h->qd_out, false);
    if (rc == MLB_OK && cudaEventRecord(h->ev1, st) != cudaSuccess) rc = MLB_ERR_CUDA;
    h->qd_ne = keep;
    if (rc != MLB_OK) return rc;
    const size_t nv = (size_t)h->n_active * (h->dtype == MLB_C128 ? 2 : 1);
    MLB_CUDA(cudaMemcpyAsync(h->qd_host, h->qd_out, (nv + 1) * 8, cudaMemcpyDeviceToHost, st));
    MLB_CUDA(cudaStreamSynchronize(st));
    float ms = 0.0f;
    MLB_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (h->qd_host[nv] != 0.0) return MLB_ERR_TIMEOUT;
    us = 1e3 * (double)ms / 20.0;
    return MLB_OK;
}

// Choose the fused column count of the handle's product (none when the
// handle has no product).  Sets h->qd_ne and the result's qd fields.
static int tune_qd(mlb_handle *h, mlb_tune_result *out) {
    if (h->precond != MLB_PRECOND_NONE || h->ew != 1) return MLB_OK;
    const bool cplx = h->dtype == MLB_C128;
    const bool narrow = h->precision == MLB_PREC_FP32_REFINED;
    const int32_t vt = cplx ? (narrow ? MLB_C64 : MLB_C128) : (narrow ? MLB_F32 : MLB_F64);
    const size_t vb = narrow ? h->esize / 2 : h->esize;
    void *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, (size_t)h->N * vb) != cudaSuccess || cudaMalloc(&y, (size_t)h->N * vb) != cudaSuccess) {
        cudaGetLastError();
        if (x) cudaFree(x);
        return MLB_ERR_OOM;
    }
    int rc = cudaMemsetAsync(x, 0, (size_t)h->N * vb, h->stream) == cudaSuccess ? MLB_OK : MLB_ERR_CUDA;
    const int def = qd_fused_columns(h->n_active, cplx, narrow);
    double def_us = 0.0, best_us = 0.0;
    int best = def;
    if (rc == MLB_OK) rc = time_qd(h, vt, def, x, y, def_us);
    best_us = def_us;
    for (int ne : {1, 2, 4}) {
        if (rc != MLB_OK) break;
        if (ne == def || ne > h->n_active || (cplx && ne > 2)) continue;
        double us = 0.0;
        rc = time_qd(h, vt, ne, x, y, us);
        if (rc == MLB_OK && us < best_us) {
            best_us = us;
            best = ne;
        }
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(x);
    cudaFree(y);
    if (rc != MLB_OK) return rc;
    h->qd_ne = best;
    out->qd_fused = best;
    out->qd_us = best_us;
    out->qd_default_us = def_us;
    return MLB_OK;
}

// Device time per iteration of `iters` iterations of A x = 1 from x = 0
// (tol 0, so exactly `iters` steps unless a breakdown ends it earlier);
// the better of two runs.
static int time_config(mlb_handle *h, int32_t iters, std::vector<char> &bh, std::vector<char> &xh, double &us) {
    mlb_result r;
    double best = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
        std::fill(xh.begin(), xh.end(), 0);
        const int rc = mlbicgstab_solve(h, bh.data(), xh.data(), 0, 0.0, iters, &r, nullptr, 0);
        if (rc != MLB_OK) return rc;
        if (r.iter > 0) best = std::min(best, 1e3 * r.kernel_ms / (double)r.iter);
    }
    us = best;
    return MLB_OK;
}

int mlbicgstab_autotune(mlb_handle *h, int32_t iters, int32_t use_cache, mlb_tune_result *out) {
    if (!h || !out || iters < 1 || iters > 100000 || (use_cache != 0 && use_cache != 1)) return MLB_ERR_ARG;
    memset(out, 0, sizeof(*out));
    MLB_CUDA(cudaSetDevice(h->device));
    const auto key = std::make_tuple(h->dtype, h->precision, h->precond, log2_floor(h->N), per_row(h), h->n_active);
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->grid = std::max(1, std::min(it->second.grid, h->grid_max));
            h->spt_cap = std::max(1, std::min(it->second.spt, (int)kConsumerWarps));
            h->qd_ne = it->second.qd_ne;
            out->grid = h->grid;
            out->spt_cap = h->spt_cap;
            out->qd_fused = h->precond == MLB_PRECOND_NONE && h->ew == 1
                                ? qd_ne_for(h, h->dtype == MLB_C128, h->precision == MLB_PREC_FP32_REFINED)
                                : 0;
            out->from_cache = 1;
            return MLB_OK;
        }
    }
    // right-hand side of ones and a zero start, in host memory
    std::vector<char> bh((size_t)h->N * h->esize, 0), xh((size_t)h->N * h->esize, 0);
    const double one = 1.0;
    for (int64_t i = 0; i < h->N; ++i) memcpy(&bh[(size_t)i * h->esize], &one, sizeof(one));
    const int g0 = h->grid, s0 = h->spt_cap;
    std::vector<int> grids, spts;
    grids.push_back(g0);
    for (int d = 1; d <= 8; d *= 2) {
        const int g = std::max(1, h->grid_want / d);
        if (std::find(grids.begin(), grids.end(), g) == grids.end()) grids.push_back(g);
    }
    spts.push_back(s0);
    for (int c : {(int)kConsumerWarps, 12, 8, 4})
        if (std::find(spts.begin(), spts.end(), c) == spts.end()) spts.push_back(c);
    double def_us = 0.0;
    int rc = time_config(h, iters, bh, xh, def_us);
    if (rc) return rc;
    int best_g = g0, best_s = s0;
    double best_us = def_us;
    int trials = 1;
    for (int g : grids)
        for (int sc : spts) {
            if (g == g0 && sc == s0) continue;
            h->grid = g;
            h->spt_cap = sc;
            double us = 0.0;
            rc = time_config(h, iters, bh, xh, us);
            ++trials;
            if (rc) {
                h->grid = g0;
                h->spt_cap = s0;
                return rc;
            }
            if (us < best_us) {
                best_us = us;
                best_g = g;
                best_s = sc;
            }
        }
    h->grid = best_g;
    h->spt_cap = best_s;
    rc = tune_qd(h, out);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = {best_g, best_s, h->qd_ne};
    }
    out->grid = best_g;
    out->spt_cap = best_s;
    out->us_per_iter = best_us;
    out->default_us_per_iter = def_us;
    out->trials = trials;
    return MLB_OK;
}

int mlbicgstab_get_tuning(const mlb_handle *h, mlb_tuning *out) {
    if (!h || !out) return MLB_ERR_ARG;
    out->grid = h->grid;
    out->spt_cap = h->spt_cap;
    out->batch_spt_cap = h->batch_spt;
    out->batch_team = h->batch_team;
    out->qd_fused = h->qd_ne;
    return MLB_OK;
}

int mlbicgstab_set_tuning(mlb_handle *h, const mlb_tuning *t) {
    if (!h || !t) return MLB_ERR_ARG;
    if (t->grid < 1 || t->grid > h->grid_max) return MLB_ERR_ARG;
    if (t->spt_cap < 1 || t->spt_cap > (int)kConsumerWarps) return MLB_ERR_ARG;
    if (t->batch_spt_cap < -1 || t->batch_spt_cap > (int)kConsumerWarps) return MLB_ERR_ARG;
    if (t->batch_team < 1 || t->batch_team > kMaxBatchTeam) return MLB_ERR_ARG;
    if (t->qd_fused != 0 && t->qd_fused != 1 && t->qd_fused != 2 && t->qd_fused != 4) return MLB_ERR_ARG;
    if (t->qd_fused == 4 && h->dtype == MLB_C128) return MLB_ERR_ARG;
    h->grid = t->grid;
    h->spt_cap = t->spt_cap;
    h->batch_spt = t->batch_spt_cap;
    h->batch_team = t->batch_team;
    h->qd_ne = t->qd_fused;
    return MLB_OK;
}

// Device time of one trial batch over `sel`: A x = 1 from x = 0 to `tol`,
// at most `maxit` iterations per system, host buffers.
static int time_batch(const std::vector<mlb_handle *> &sel, double tol_, int64_t maxit, double &ms) {
    const size_t cnt = sel.size();
    std::vector<std::vector<char>> bh(cnt), xh(cnt);
    std::vector<const void *> bp(cnt);
    std::vector<void *> xp(cnt);
    std::vector<double> tol(cnt, tol_);
    std::vector<int64_t> its(cnt, maxit);
    std::vector<mlb_result> res(cnt);
    const double one = 1.0;
    for (size_t s = 0; s < cnt; ++s) {
        const mlb_handle *h = sel[s];
        bh[s].assign((size_t)h->N * h->esize, 0);
        xh[s].assign((size_t)h->N * h->esize, 0);
        for (int64_t i = 0; i < h->N; ++i) memcpy(&bh[s][(size_t)i * h->esize], &one, sizeof(one));
        bp[s] = bh[s].data();
        xp[s] = xh[s].data();
    }
    const int rc = mlbicgstab_solve_batch(sel.data(), (int32_t)cnt, bp.data(), xp.data(), 0, tol.data(), its.data(),
                                          res.data());
    if (rc != MLB_OK) return rc;
    ms = res[0].kernel_ms;
    return MLB_OK;
}

int mlbicgstab_autotune_batch(mlb_handle *const *hs, int32_t count, double tol, int64_t maxit, int32_t use_cache,
                              mlb_batch_tune_result *out) {
    if (!hs || count <= 0 || !out || !(tol >= 0.0) || maxit < 1 || maxit > 10000000 ||
        (use_cache != 0 && use_cache != 1))
        return MLB_ERR_ARG;
    memset(out, 0, sizeof(*out));
    for (int32_t s = 0; s < count; ++s) {
        const mlb_handle *h = hs[s];
        if (!h || h->dtype != hs[0]->dtype || h->precision != hs[0]->precision || h->device != hs[0]->device)
            return MLB_ERR_ARG;
        for (int32_t t = 0; t < s; ++t)
            if (hs[t] == h) return MLB_ERR_ARG;   // each system needs its own handle
        if (h->ew != 1) return MLB_ERR_UNSUPPORTED;
    }
    std::vector<mlb_handle *> all(hs, hs + count);
    int64_t ntot = 0;
    for (mlb_handle *h : all) ntot += h->N;
    // size classes in a fixed order
    std::map<std::pair<int, int64_t>, std::vector<mlb_handle *>> classes;
    for (mlb_handle *h : all) classes[{log2_floor(h->N), per_row(h)}].push_back(h);
    out->classes = (int32_t)classes.size();
    double ms = 0.0;
    int trials = 0;
    int rc = time_batch(all, tol, maxit, ms);
    ++trials;
    if (rc) return rc;
    out->default_ms = ms;
    // team size, on the whole trial batch
    const mlb_handle *h0 = all[0];
    const auto tkey = std::make_tuple(h0->dtype, h0->precision, h0->precond, (int)count, log2_floor(ntot));
    int team = -1;
    bool team_cached = false;
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_bteam_cache.find(tkey);
        if (it != g_bteam_cache.end()) {
            team = it->second;
            team_cached = true;
        }
    }
    if (team < 0) {
        std::vector<int> cand{all[0]->batch_team};
        for (int c : {1, 2, 4, 8})
            if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
        double best_ms = 1e300;
        for (int c : cand) {
            for (mlb_handle *h : all) h->batch_team = c;
            double t = 0.0;
            rc = time_batch(all, tol, maxit, t);
            ++trials;
            if (rc) return rc;
            if (t < best_ms) {
                best_ms = t;
                team = c;
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_bteam_cache[tkey] = team;
    }
    for (mlb_handle *h : all) h->batch_team = team;
    out->team = team;
    // tile caps per size class
    for (auto &kv : classes) {
        std::vector<mlb_handle *> &sel = kv.second;
        const mlb_handle *hc = sel[0];
        const auto key = std::make_tuple(hc->dtype, hc->precision, hc->precond, kv.first.first, kv.first.second);
        if (use_cache) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_btune_cache.find(key);
            if (it != g_btune_cache.end()) {
                for (mlb_handle *h : sel) h->batch_spt = it->second;
                ++out->from_cache;
                continue;
            }
        }
        std::vector<int> caps{batch_cap(hc)};
        for (int c : {(int)kConsumerWarps, 12, 8, 4, 0})
            if (std::find(caps.begin(), caps.end(), c) == caps.end()) caps.push_back(c);
        std::vector<int> keep;
        for (mlb_handle *h : sel) keep.push_back(h->batch_spt);
        int best = caps[0];
        double best_ms = 1e300;
        for (int c : caps) {
            for (mlb_handle *h : sel) h->batch_spt = c;
            double t = 0.0;
            rc = time_batch(sel, tol, maxit, t);
            ++trials;
            if (rc != MLB_OK) {
                for (size_t i = 0; i < sel.size(); ++i) sel[i]->batch_spt = keep[i];
                return rc;
            }
            if (t < best_ms) {
                best_ms = t;
                best = c;
            }
        }
        for (mlb_handle *h : sel) h->batch_spt = best;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_btune_cache[key] = best;
    }
    out->trials = team_cached && out->from_cache == out->classes ? 0 : trials;
    rc = time_batch(all, tol, maxit, ms);
    if (rc) return rc;
    out->tuned_ms = ms;
    return MLB_OK;
}

int mlbicgstab_set_n(mlb_handle *h, int32_t n) {
    if (!h || n < 1 || n > h->n) return MLB_ERR_ARG;
    h->n_active = n;
    return MLB_OK;
}

int32_t mlbicgstab_next_n(int32_t n, double t_prev, double t_cur, int32_t step, int32_t n_min, int32_t n_max) {
    if (step < 0 || n_min < 1 || n_max < n_min || n < n_min || n > n_max) return -1;
    int64_t m = t_prev > t_cur ? (int64_t)n + step : (int64_t)n - step;
    if (m < n_min) m = n_min;
    if (m > n_max) m = n_max;
    return (int32_t)m;
}

int mlbicgstab_solve_sequence(mlb_handle *const *hs, int32_t count, const void *const *b, void *const *x,
                              int32_t on_device, const double *tol, const int64_t *maxit,
                              const mlb_sequence_options *so, mlb_result *res, int32_t *n_used) {
    if (!hs || count <= 0 || !b || !x || !tol || !maxit || !so || !res || !n_used) return MLB_ERR_ARG;
    if (so->step < 0 || so->n_min < 1 || so->n_max < so->n_min || so->n0 < so->n_min || so->n0 > so->n_max)
        return MLB_ERR_ARG;
    for (int32_t s = 0; s < count; ++s)
        if (!hs[s] || hs[s]->n < so->n_max) return MLB_ERR_ARG;
    // every handle gets its n back at the end
    std::vector<std::pair<mlb_handle *, int>> saved;
    for (int32_t s = 0; s < count; ++s) {
        bool seen = false;
        for (auto &p : saved) seen = seen || p.first == hs[s];
        if (!seen) saved.push_back({hs[s], hs[s]->n_active});
    }
    int rc = MLB_OK;
    int32_t n = so->n0;
    double t_prev = 0.0;
    for (int32_t s = 0; s < count; ++s) {
        hs[s]->n_active = n;
        n_used[s] = n;
        rc = mlbicgstab_solve(hs[s], b[s], x[s], on_device, tol[s], maxit[s], &res[s], nullptr, 0);
        if (rc != MLB_OK) break;
        const double t = res[s].kernel_ms;
        if (s >= 1) n = mlbicgstab_next_n(n, t_prev, t, so->step, so->n_min, so->n_max);
        t_prev = t;
    }
    for (auto &p : saved) p.first->n_active = p.second;
    return rc;
}


int mlbicgstab_spmv_qdot(mlb_handle *h, const void *x, void *y, void *d) {
    if (!h || !x || !y || !d) return MLB_ERR_ARG;
    if (h->precond != MLB_PRECOND_NONE || h->ew != 1) return MLB_ERR_UNSUPPORTED;
    MLB_CUDA(cudaSetDevice(h->device));
    if (!is_device_ptr(x, h->device) || !is_device_ptr(y, h->device)) return MLB_ERR_ARG;
    cudaStream_t st = h->stream;
    const bool cplx = h->dtype == MLB_C128;
    if (int rc = qd_enqueue(h, cplx ? MLB_C128 : MLB_F64, x, y, h->qd_out, true)) return rc;
    MLB_CUDA(cudaEventRecord(h->ev1, st));
    // d and the status flag behind it in one copy, through pinned memory
    const size_t nv = (size_t)h->n_active * (cplx ? 2 : 1);
    MLB_CUDA(cudaMemcpyAsync(h->qd_host, h->qd_out, (nv + 1) * 8, cudaMemcpyDeviceToHost, st));
    MLB_CUDA(cudaStreamSynchronize(st));
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->qd_ms = ms;
    cudaGetLastError();
    if (h->qd_host[nv] != 0.0) return MLB_ERR_TIMEOUT;
    memcpy(d, h->qd_host, nv * 8);
    return MLB_OK;
}

int mlbicgstab_spmv_qdot_async(mlb_handle *h, int32_t value_type, const void *x, void *y, void *d) {
    if (!h || !x || !y || !d) return MLB_ERR_ARG;
    if (h->precond != MLB_PRECOND_NONE || h->ew != 1) return MLB_ERR_UNSUPPORTED;
    MLB_CUDA(cudaSetDevice(h->device));
    if (!is_device_ptr(x, h->device) || !is_device_ptr(y, h->device) || !is_device_ptr(d, h->device))
        return MLB_ERR_ARG;
    return qd_enqueue(h, value_type, x, y, (double *)d, false);
}

int mlbicgstab_selftest_barrier_timeout(int32_t grid, int64_t timeout_ns) {
    if (grid < 1 || grid > 64 || timeout_ns <= 0 || timeout_ns > 10000000000LL) return MLB_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    BarrierState *bs = nullptr;
    MLB_CUDA(cudaMalloc(&bs, sizeof(BarrierState)));
    cudaError_t e = cudaMemset(bs, 0, sizeof(BarrierState));
    if (e == cudaSuccess) e = launch_barrier_selftest(grid, bs, (uint64_t)timeout_ns, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    BarrierState hb;
    memset(&hb, 0, sizeof(hb));
    if (e == cudaSuccess) e = cudaMemcpy(&hb, bs, sizeof(hb), cudaMemcpyDeviceToHost);
    cudaFree(bs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLB_ERR_CUDA;
    }
    return hb.status == kStatusTimeout ? MLB_ERR_TIMEOUT : MLB_OK;
}

}  // extern "C"
