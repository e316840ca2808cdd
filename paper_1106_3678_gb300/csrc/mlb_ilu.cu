// Host side of the ILU(0) preconditioner (Algorithm 7.1 with M = L U; the
// paper's experiments precondition with ILU(0), §5): the factors in A's
// pattern, the level sets of the two triangular solves, and M^{-H} v for
// the setup product F = M^{-H} A^H Q.  The triangular solves of the
// iteration run on the device (Engine::ilu_solve).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <utility>

#include "mlb_internal.h"

namespace mlb {
namespace {

inline double cj(double v) { return v; }
inline std::complex<double> cj(std::complex<double> v) { return std::conj(v); }

// Rows grouped by level: level(i) = 1 + the largest level among the rows
// row i reads (0 if none), rows ascending within a level.
void group_levels(const std::vector<int32_t> &lev, int nlev, std::vector<int32_t> &rows,
                  std::vector<int32_t> &ptr) {
    ptr.assign(nlev + 1, 0);
    for (int32_t l : lev) ptr[l + 1]++;
    for (int l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
    rows.assign(lev.size(), 0);
    std::vector<int32_t> next(ptr.begin(), ptr.end() - 1);
    for (size_t i = 0; i < lev.size(); ++i) rows[next[lev[i]]++] = (int32_t)i;
}

template <typename V>
int build_t(const mlb_matrix *A, IluHost &f) {
    const int64_t N = A->nrows;
    const V *a = (const V *)A->values;
    // A's pattern with columns increasing in each row; repeated entries of
    // a row are one entry (their sum)
    f.rp.assign(N + 1, 0);
    f.dpos.assign(N, -1);
    std::vector<int32_t> ci;
    std::vector<V> val;
    ci.reserve(A->nnz);
    val.reserve(A->nnz);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int64_t r = 0; r < N; ++r) {
        row.clear();
        for (int64_t k = A->row_ptr[r]; k < A->row_ptr[r + 1]; ++k) row.emplace_back(A->col_idx[k], k);
        std::stable_sort(row.begin(), row.end(),
                         [](const std::pair<int32_t, int64_t> &p, const std::pair<int32_t, int64_t> &q) {
                             return p.first < q.first;
                         });
        const int64_t start = (int64_t)ci.size();
        for (const auto &e : row) {
            if ((int64_t)ci.size() > start && ci.back() == e.first) {
                val.back() += a[e.second];
            } else {
                ci.push_back(e.first);
                val.push_back(a[e.second]);
            }
        }
        for (int64_t k = start; k < (int64_t)ci.size(); ++k)
            if (ci[k] == r) f.dpos[r] = (int32_t)(k - start);
        if (f.dpos[r] < 0) return MLB_ERR_ARG;   // ILU(0) needs a stored diagonal
        f.rp[r + 1] = (int64_t)ci.size();
    }
    // elimination restricted to the pattern, one row at a time: for each
    // k < i stored in row i (increasing k), l_ik = a_ik / u_kk, then
    // a_ij -= l_ik u_kj for the j > k stored in both rows i and k
    std::vector<int64_t> at(N, -1);   // position of column j in the current row
    int rc = MLB_OK;
    for (int64_t i = 0; i < N && rc == MLB_OK; ++i) {
        const int64_t r0 = f.rp[i], r1 = f.rp[i + 1], di = r0 + f.dpos[i];
        for (int64_t k = r0; k < r1; ++k) at[ci[k]] = k;
        for (int64_t p = r0; p < di; ++p) {
            const int64_t k = ci[p];
            const int64_t dk = f.rp[k] + f.dpos[k];
            val[p] = val[p] / val[dk];
            const V lik = val[p];
            for (int64_t q = dk + 1; q < f.rp[k + 1]; ++q) {
                const int64_t t = at[ci[q]];
                if (t >= 0) val[t] -= lik * val[q];
            }
        }
        for (int64_t k = r0; k < r1; ++k) at[ci[k]] = -1;
        // a zero or non-finite pivot has no ILU(0)
        if (!(std::abs(val[di]) > 0.0) || !std::isfinite(std::abs(val[di]))) rc = MLB_ERR_ARG;
    }
    if (rc) return rc;
    for (const V &v : val)
        if (!std::isfinite(std::abs(v))) return MLB_ERR_ARG;
    f.ci = std::move(ci);
    f.lu.assign((const char *)val.data(), (const char *)(val.data() + val.size()));
    f.nnz = (int64_t)val.size();
    // level sets: L from the first row down, U from the last row up
    std::vector<int32_t> lev(N, 0);
    int nl = 0;
    for (int64_t i = 0; i < N; ++i) {
        int32_t l = 0;
        for (int64_t k = f.rp[i]; k < f.rp[i] + f.dpos[i]; ++k) l = std::max(l, lev[f.ci[k]] + 1);
        lev[i] = l;
        nl = std::max(nl, l + 1);
    }
    group_levels(lev, nl, f.lrows, f.lptr);
    f.nlev_l = nl;
    int nu = 0;
    for (int64_t i = N - 1; i >= 0; --i) {
        int32_t l = 0;
        for (int64_t k = f.rp[i] + f.dpos[i] + 1; k < f.rp[i + 1]; ++k) l = std::max(l, lev[f.ci[k]] + 1);
        lev[i] = l;
        nu = std::max(nu, l + 1);
    }
    group_levels(lev, nu, f.urows, f.uptr);
    f.nlev_u = nu;
    // level-position copies (kIluEll entries per row, zero padded)
    const V *lu = (const V *)f.lu.data();
    f.lcnt.assign(N, 0);
    f.ucnt.assign(N, 0);
    f.lell_c.assign((size_t)kIluEll * N, 0);
    f.uell_c.assign((size_t)kIluEll * N, 0);
    std::vector<V> la((size_t)kIluEll * N, V(0)), ua((size_t)kIluEll * N, V(0)), ud(N, V(0));
    for (int64_t q = 0; q < N; ++q) {
        const int64_t i = f.lrows[q], k0 = f.rp[i], d = k0 + f.dpos[i];
        f.lcnt[q] = (int32_t)(d - k0);
        for (int64_t e = 0; e < kIluEll && k0 + e < d; ++e) {
            f.lell_c[e * N + q] = f.ci[k0 + e];
            la[e * N + q] = lu[k0 + e];
        }
        const int64_t j = f.urows[q], dj = f.rp[j] + f.dpos[j], k1 = f.rp[j + 1];
        f.ucnt[q] = (int32_t)(k1 - dj - 1);
        for (int64_t e = 0; e < kIluEll && dj + 1 + e < k1; ++e) {
            f.uell_c[e * N + q] = f.ci[dj + 1 + e];
            ua[e * N + q] = lu[dj + 1 + e];
        }
        ud[q] = lu[dj];
    }
    auto bytes = [](const std::vector<V> &x, std::vector<char> &out) {
        out.assign((const char *)x.data(), (const char *)(x.data() + x.size()));
    };
    bytes(la, f.lell_a);
    bytes(ua, f.uell_a);
    bytes(ud, f.udiag);
    return MLB_OK;
}

// v <- M^{-H} v with M^H = U^H L^H: U^H t = v (U^H is lower triangular;
// row i of U is column i of U^H), then L^H v = t (unit upper triangular).
template <typename V>
void apply_h_t(const IluHost &f, V *v) {
    const int64_t N = (int64_t)f.rp.size() - 1;
    const V *lu = (const V *)f.lu.data();
    for (int64_t i = 0; i < N; ++i) {
        const int64_t d = f.rp[i] + f.dpos[i];
        v[i] = v[i] / cj(lu[d]);
        const V vi = v[i];
        for (int64_t k = d + 1; k < f.rp[i + 1]; ++k) v[f.ci[k]] -= cj(lu[k]) * vi;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        const V vi = v[i];
        for (int64_t k = f.rp[i]; k < f.rp[i] + f.dpos[i]; ++k) v[f.ci[k]] -= cj(lu[k]) * vi;
    }
}

}  // namespace

int mc_order(const mlb_matrix *A, std::vector<int32_t> &perm) {
    const int64_t N = A->nrows;
    // transposed pattern (who lists column i), for the symmetrised graph
    std::vector<int64_t> tp(N + 1, 0);
    for (int64_t k = 0; k < A->nnz; ++k) tp[A->col_idx[k] + 1]++;
    for (int64_t r = 0; r < N; ++r) tp[r + 1] += tp[r];
    std::vector<int32_t> tr(A->nnz);
    {
        std::vector<int64_t> next(tp.begin(), tp.end() - 1);
        for (int64_t r = 0; r < N; ++r)
            for (int64_t k = A->row_ptr[r]; k < A->row_ptr[r + 1]; ++k) tr[next[A->col_idx[k]]++] = (int32_t)r;
    }
    std::vector<int32_t> color(N, -1);
    std::vector<int64_t> seen;   // seen[c] == i: colour c is taken by a neighbour of row i
    int ncolors = 0;
    for (int64_t i = 0; i < N; ++i) {
        auto mark = [&](int64_t j) {
            if (j != i && color[j] >= 0) {
                if ((size_t)color[j] >= seen.size()) seen.resize(color[j] + 1, -1);
                seen[color[j]] = i;
            }
        };
        for (int64_t k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) mark(A->col_idx[k]);
        for (int64_t k = tp[i]; k < tp[i + 1]; ++k) mark(tr[k]);
        int c = 0;
        while ((size_t)c < seen.size() && seen[c] == i) ++c;
        color[i] = c;
        ncolors = std::max(ncolors, c + 1);
    }
    // colour by colour, natural order within a colour (a stable counting sort)
    std::vector<int64_t> start(ncolors + 1, 0);
    for (int64_t i = 0; i < N; ++i) start[color[i] + 1]++;
    for (int c = 0; c < ncolors; ++c) start[c + 1] += start[c];
    perm.assign(N, 0);
    for (int64_t i = 0; i < N; ++i) perm[start[color[i]]++] = (int32_t)i;
    return ncolors;
}

void permute_csr(const mlb_matrix *A, const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm,
                 size_t es, std::vector<int64_t> &rp, std::vector<int32_t> &ci, std::vector<char> &val) {
    const int64_t N = A->nrows;
    rp.assign(N + 1, 0);
    for (int64_t r = 0; r < N; ++r) {
        const int64_t o = perm[r];
        rp[r + 1] = rp[r] + (A->row_ptr[o + 1] - A->row_ptr[o]);
    }
    ci.assign(A->nnz, 0);
    val.assign((size_t)A->nnz * es, 0);
    const char *av = (const char *)A->values;
    for (int64_t r = 0; r < N; ++r) {
        const int64_t o = perm[r];
        int64_t d = rp[r];
        for (int64_t k = A->row_ptr[o]; k < A->row_ptr[o + 1]; ++k, ++d) {
            ci[d] = iperm[A->col_idx[k]];
            memcpy(&val[(size_t)d * es], av + (size_t)k * es, es);
        }
    }
}

int ilu0_build(const mlb_matrix *A, IluHost &out) {
    return A->dtype == MLB_C128 ? build_t<std::complex<double>>(A, out) : build_t<double>(A, out);
}

void ilu0_apply_h(const IluHost &f, bool cplx, void *v) {
    if (cplx) apply_h_t(f, (std::complex<double> *)v);
    else apply_h_t(f, (double *)v);
}

}  // namespace mlb
