/*
 * Body of the CPU oracle, compiled twice by mlb_oracle.c: once with
 * S = double (suffix _d) and once with S = double complex (suffix _z).
 * TEST INFRASTRUCTURE ONLY (see the header of mlb_oracle.c).
 *
 * Every vector operation is one plain sequential loop (the multi-core
 * build, ORC_PAR, shares elementwise loops among threads and takes inner
 * products and norms over fixed blocks; see below).  Inner products
 * conjugate their left argument, u^H v = sum_i conj(u_i) v_i, as the paper's
 * ^H does; norms are sqrt(sum_i |v_i|^2).
 */

/* ---- vector primitives (one Table 4.3 operation each) ------------------ */

#ifndef ORC_PAR
/* u^H v: one "dot product" of Table 4.3. */
static S SFX(dot)(int64_t N, const S *u, const S *v, int64_t *ops)
{
    S s = 0;
    for (int64_t i = 0; i < N; ++i)
        s += CONJ(u[i]) * v[i];
    ops[ORC_OP_DOT]++;
    return s;
}

/* ||v||_2, used by the stopping rule of §5 (not a Table 4.3 entry). */
static double SFX(nrm2)(int64_t N, const S *v, int64_t *ops)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i)
        s += ABS2(v[i]);
    ops[ORC_OP_NORM]++;
    return sqrt(s);
}
#else
/* Multi-core build: the same sums taken over fixed blocks of ORC_BLOCK
 * consecutive entries (each block summed in index order, then the block
 * sums in block order), the blocks shared among threads.  The block
 * partition does not depend on the thread count, so results are identical
 * for every thread count; they differ from the sequential sums above only
 * in rounding order. */
#define ORC_BLOCK 1024
static S SFX(dot)(int64_t N, const S *u, const S *v, int64_t *ops)
{
    const int64_t nb = (N + ORC_BLOCK - 1) / ORC_BLOCK;
    S *part = (S *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(S));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t i1 = (b + 1) * ORC_BLOCK < N ? (b + 1) * ORC_BLOCK : N;
        S t = 0;
        for (int64_t i = b * ORC_BLOCK; i < i1; ++i)
            t += CONJ(u[i]) * v[i];
        part[b] = t;
    }
    S s = 0;
    for (int64_t b = 0; b < nb; ++b)
        s += part[b];
    free(part);
    ops[ORC_OP_DOT]++;
    return s;
}

static double SFX(nrm2)(int64_t N, const S *v, int64_t *ops)
{
    const int64_t nb = (N + ORC_BLOCK - 1) / ORC_BLOCK;
    double *part = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t i1 = (b + 1) * ORC_BLOCK < N ? (b + 1) * ORC_BLOCK : N;
        double t = 0.0;
        for (int64_t i = b * ORC_BLOCK; i < i1; ++i)
            t += ABS2(v[i]);
        part[b] = t;
    }
    double s = 0.0;
    for (int64_t b = 0; b < nb; ++b)
        s += part[b];
    free(part);
    ops[ORC_OP_NORM]++;
    return sqrt(s);
}
#endif

/* y = A x for CSR A: y_r = sum_k a_{r,col(k)} x_{col(k)} (row order). */
static void SFX(csr_apply)(int64_t N, const int64_t *rp, const int32_t *ci,
                           const S *av, const S *x, S *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < N; ++r) {
        S s = 0;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
            s += av[k] * x[ci[k]];
        y[r] = s;
    }
}

/* One "matvec A v" of Table 4.3. */
static void SFX(matvec)(int64_t N, const int64_t *rp, const int32_t *ci,
                        const S *av, const S *x, S *y, int64_t *ops)
{
    SFX(csr_apply)(N, rp, ci, av, x, y);
    ops[ORC_OP_MATVEC]++;
}

/* y <- y + a x : one "saxpy". */
static void SFX(axpy)(int64_t N, S a, const S *x, S *y, int64_t *ops)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        y[i] = y[i] + a * x[i];
    ops[ORC_OP_SAXPY]++;
}

/* out <- x + a y (out may alias y) : one "saxpy". */
static void SFX(xpay)(int64_t N, const S *x, S a, const S *y, S *out,
                      int64_t *ops)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        out[i] = x[i] + a * y[i];
    ops[ORC_OP_SAXPY]++;
}

/* y <- a y : one "alpha v" of Table 4.3. */
static void SFX(scal)(int64_t N, S a, S *y, int64_t *ops)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        y[i] = a * y[i];
    ops[ORC_OP_SCALE]++;
}

/* g <- z - g / omega (the omega-correction of Algorithm 7.1, division as
 * written there) : counted as one "saxpy". */
static void SFX(omega_corr)(int64_t N, const S *z, S omega, S *g, int64_t *ops)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        g[i] = z[i] - g[i] / omega;
    ops[ORC_OP_SAXPY]++;
}

/* ---- public entry points ------------------------------------------------ */

/* y = A x (definition of the sparse product). */
void SFX(orc_spmv)(int64_t N, const int64_t *rp, const int32_t *ci,
                   const S *av, const S *x, S *y)
{
    SFX(csr_apply)(N, rp, ci, av, x, y);
}

/* F = A^H Q(:, 0:m-1): column s is sum_r conj(a_{r,c}) q_s(r) placed at c,
 * i.e. the definition of the conjugate-transposed product, taken entry by
 * entry of A (Algorithm 4.1, step 2; M = I in Algorithm 7.1, step 2).
 * Q and F are column-major with leading dimension N; F is overwritten. */
void SFX(orc_ahq)(int64_t N, const int64_t *rp, const int32_t *ci,
                  const S *av, int32_t m, const S *Q, S *F)
{
    for (int64_t t = 0; t < (int64_t)m * N; ++t)
        F[t] = 0;
    for (int32_t s = 0; s < m; ++s) {
        const S *q = Q + (int64_t)s * N;
        S *f = F + (int64_t)s * N;
        for (int64_t r = 0; r < N; ++r)
            for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
                f[ci[k]] += CONJ(av[k]) * q[r];
    }
}

/*
 * ILU(0), the preconditioner of the paper's experiments (§5): L unit lower
 * triangular and U upper triangular, both with the sparsity pattern of A,
 * such that (L U)_ij = a_ij for every (i, j) in that pattern.  Computed by
 * the textbook row-oriented elimination restricted to the pattern (Saad,
 * Iterative Methods for Sparse Linear Systems, 2nd ed., Algorithm 10.4):
 * for each row i and each k < i of its pattern in increasing order,
 * a_ik <- a_ik / a_kk, then a_ij <- a_ij - a_ik a_kj for every j > k that
 * is in the pattern of both row i and row k.
 *
 * In: CSR A, column indices increasing within each row, a stored diagonal
 * entry in every row.  Out: lu (the nnz values in A's pattern: strictly
 * lower part = L without its unit diagonal, the rest = U) and dpos[r] =
 * position of row r's diagonal.  Returns 0; -1 when a row is unsorted or
 * has no diagonal; -3 when a pivot u_kk is zero; -2 on allocation failure.
 */
int SFX(orc_ilu0)(int64_t N, const int64_t *rp, const int32_t *ci, const S *av,
                  S *lu, int64_t *dpos)
{
    for (int64_t r = 0; r < N; ++r) {
        dpos[r] = -1;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
            if (k > rp[r] && ci[k] <= ci[k - 1])
                return -1;
            if (ci[k] == r)
                dpos[r] = k;
        }
        if (dpos[r] < 0)
            return -1;
    }
    for (int64_t k = 0; k < rp[N]; ++k)
        lu[k] = av[k];
    int64_t *pos = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    if (!pos)
        return -2;
    for (int64_t t = 0; t < N; ++t)
        pos[t] = -1;
    int rc = 0;
    for (int64_t i = 0; i < N && rc == 0; ++i) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            pos[ci[k]] = k;
        for (int64_t ik = rp[i]; ik < dpos[i]; ++ik) {
            const int64_t k = ci[ik];
            const S ukk = lu[dpos[k]];
            if (ukk == 0) {
                rc = -3;
                break;
            }
            lu[ik] = lu[ik] / ukk;
            for (int64_t kj = dpos[k] + 1; kj < rp[k + 1]; ++kj) {
                const int64_t ij = pos[ci[kj]];
                if (ij >= 0)
                    lu[ij] = lu[ij] - lu[ik] * lu[kj];
            }
        }
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            pos[ci[k]] = -1;
    }
    free(pos);
    for (int64_t i = 0; i < N && rc == 0; ++i)
        if (lu[dpos[i]] == 0)
            rc = -3;
    return rc;
}

/* The preconditioner M of Algorithm 7.1 handed to the oracle: none, a
 * diagonal (mdiag), or ILU(0) factors in A's pattern (lu, dpos). */
typedef struct {
    int64_t N;
    const int64_t *rp;
    const int32_t *ci;
    const S *mdiag;
    const S *lu;
    const int64_t *dpos;
} SFX(pc_t);

/* dst = M^{-1} src.  Diagonal: elementwise division.  ILU(0): L y = src
 * by forward substitution, then U dst = y by backward substitution (rows
 * in order, each a plain sequential sum). */
static void SFX(minv)(const SFX(pc_t) *pc, const S *src, S *dst)
{
    const int64_t N = pc->N;
    if (pc->mdiag) {
        const S *mdiag = pc->mdiag;
        for (int64_t t = 0; t < N; ++t)
            dst[t] = src[t] / mdiag[t];
        return;
    }
    const int64_t *rp = pc->rp, *dp = pc->dpos;
    const int32_t *ci = pc->ci;
    const S *lu = pc->lu;
    for (int64_t i = 0; i < N; ++i) {
        S s = src[i];
        for (int64_t k = rp[i]; k < dp[i]; ++k)
            s -= lu[k] * dst[ci[k]];
        dst[i] = s;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        S s = dst[i];
        for (int64_t k = dp[i] + 1; k < rp[i + 1]; ++k)
            s -= lu[k] * dst[ci[k]];
        dst[i] = s / lu[dp[i]];
    }
}

/* v <- M^{-H} v (for F = M^{-H} A^H Q).  Diagonal: division by conj(m).
 * ILU(0): M^H = U^H L^H, so first U^H t = v (U^H is lower triangular:
 * forward, column by column of U^H, i.e. row by row of U), then
 * L^H v = t (unit upper: backward, row by row of L). */
static void SFX(minv_h)(const SFX(pc_t) *pc, S *v)
{
    const int64_t N = pc->N;
    if (pc->mdiag) {
        const S *mdiag = pc->mdiag;
        for (int64_t t = 0; t < N; ++t)
            v[t] = v[t] / CONJ(mdiag[t]);
        return;
    }
    const int64_t *rp = pc->rp, *dp = pc->dpos;
    const int32_t *ci = pc->ci;
    const S *lu = pc->lu;
    for (int64_t i = 0; i < N; ++i) {
        v[i] = v[i] / CONJ(lu[dp[i]]);
        for (int64_t k = dp[i] + 1; k < rp[i + 1]; ++k)
            v[ci[k]] -= CONJ(lu[k]) * v[i];
    }
    for (int64_t i = N - 1; i >= 0; --i)
        for (int64_t k = rp[i]; k < dp[i]; ++k)
            v[ci[k]] -= CONJ(lu[k]) * v[i];
}

/* The two applications, exported for the pins. */
void SFX(orc_minv)(int64_t N, const int64_t *rp, const int32_t *ci, const S *mdiag,
                   const S *lu, const int64_t *dpos, const S *src, S *dst)
{
    SFX(pc_t) pc = {N, rp, ci, mdiag, lu, dpos};
    SFX(minv)(&pc, src, dst);
}
void SFX(orc_minv_h)(int64_t N, const int64_t *rp, const int32_t *ci, const S *mdiag,
                     const S *lu, const int64_t *dpos, S *v)
{
    SFX(pc_t) pc = {N, rp, ci, mdiag, lu, dpos};
    SFX(minv_h)(&pc, v);
}

/*
 * ML(n)BiCGStabt: Algorithm 7.1 of the paper with M = I, which is
 * Algorithm 4.1 with its k-loop split into k = jn + i, 1 <= i <= n, j >= 0
 * (§2, eq. 2.1).  Stopping rule ||r_k||_2/||b||_2 < tol on the recursive
 * residual after every update of r (and of u), ||b|| replaced by 1 when
 * b = 0 (§5); flags 0 = converged, 1 = iteration limit, -1 = breakdown
 * (c = 0, ||A u|| = 0 or omega = 0).  Eq. 5.1 (kappa > 0) guards omega.
 *
 * Storage (the "ring"): g_k, w_k, c_k of iterate k = jn + s live in slot
 * s = k mod n of G, W, c.  While step jn+i runs, slots 0..i-1 hold block j
 * and slots i..n-1 still hold block j-1, which is exactly what steps 10-17
 * of Algorithm 7.1 read; slot i is then overwritten in place.
 *
 * Preconditioning (Algorithm 7.1 with M != I): mdiag, when not NULL, is
 * the diagonal of M; ilu and ilu_dpos, when not NULL, are the ILU(0)
 * factors of A from orc_ilu0 (M = L U).  Right preconditioning: as written in the
 * algorithm: F = M^{-H} A^H Q (step 2), g^ = M^{-1} g is kept beside every
 * g (steps 2, 31, 50) and is what x advances along (steps 6, 35) and what
 * A multiplies (w = A g^); u^ = M^{-1} u (step 37) gives z = A u^ and
 * x += omega u^ (steps 38-39); the guard of Eq. 5.1 is taken with A u^ in
 * place of A u.  With neither given, M = I: no g^ is formed and the
 * arithmetic is exactly that of Algorithm 4.1.
 *
 * Inputs: CSR A (N rows), Q (N x n, column-major, ld N), b, x (in: x_0,
 * out: solution).  Optional histories (NULL to skip):
 *   err_hist[k]       relative residual after iteration k (k = 0: initial)
 *   x_hist[(k-1)*N..] x after iteration k, for k <= x_cap
 *   blk_ops[5*j..]    operation counters when block j starts
 *   trace[2*(k-1)..]  (j, i) of iteration k
 * Returns 0, or -2 on allocation failure.
 */
int SFX(orc_mlbicgstabt)(int64_t N, const int64_t *rp, const int32_t *ci,
                         const S *av, int32_t n, const S *Q, const S *b,
                         S *x, int64_t maxit, double tol, double kappa,
                         const S *mdiag, const S *ilu, const int64_t *ilu_dpos,
                         orc_result *res,
                         double *err_hist, int64_t err_cap,
                         S *x_hist, int64_t x_cap,
                         int64_t *blk_ops, int64_t blk_cap,
                         int32_t *trace, int64_t trace_cap)
{
    int64_t *ops = res->ops;
    memset(res, 0, sizeof(*res));
    res->flag = 1;

    S *G = (S *)calloc((size_t)N * n, sizeof(S));
    S *W = (S *)calloc((size_t)N * n, sizeof(S));
    S *F = n > 1 ? (S *)calloc((size_t)N * (n - 1), sizeof(S)) : NULL;
    S *r = (S *)calloc((size_t)N, sizeof(S));
    S *z = (S *)calloc((size_t)N, sizeof(S));
    S *c = (S *)calloc((size_t)n, sizeof(S));
    /* g^ slots and u^ (M != I only; with M = I they are G and r) */
    const SFX(pc_t) pc = {N, rp, ci, mdiag, ilu, ilu_dpos};
    const int pc_on = mdiag || ilu;
    S *Gh = pc_on ? (S *)calloc((size_t)N * n, sizeof(S)) : G;
    S *uh = pc_on ? (S *)calloc((size_t)N, sizeof(S)) : r;
    if (!G || !W || (n > 1 && !F) || !r || !z || !c || !Gh || !uh) {
        free(G); free(W); free(F); free(r); free(z); free(c);
        if (pc_on) { free(Gh); free(uh); }
        return -2;
    }

    int64_t iter = 0;
    int64_t j = 0;
    int32_t i = 0;
    double err;
    S e, alpha, omega = 0;

#define RECORD()                                                              \
    do {                                                                      \
        if (err_hist && iter < err_cap) err_hist[iter] = err;                 \
        if (x_hist && iter >= 1 && iter <= x_cap)                             \
            memcpy(x_hist + (iter - 1) * N, x, (size_t)N * sizeof(S));        \
        if (trace && iter >= 1 && iter <= trace_cap) {                        \
            trace[2 * (iter - 1)] = (int32_t)j;                               \
            trace[2 * (iter - 1) + 1] = i;                                    \
        }                                                                     \
    } while (0)

    /* stopping-rule denominator */
    double bnrm2 = SFX(nrm2)(N, b, ops);
    if (bnrm2 == 0.0)
        bnrm2 = 1.0;

    /* step 2: r_0 = b - A x_0 */
    SFX(matvec)(N, rp, ci, av, x, r, ops);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < N; ++t)
        r[t] = b[t] - r[t];
    err = SFX(nrm2)(N, r, ops) / bnrm2;
    RECORD();
    if (err < tol) {
        res->flag = 0;
        goto done;
    }

    /* step 2: [f_1..f_{n-1}] = M^{-H} A^H [q_1..q_{n-1}] */
    if (n > 1) {
        SFX(orc_ahq)(N, rp, ci, av, n - 1, Q, F);
        if (pc_on)
            for (int32_t s = 0; s < n - 1; ++s)
                SFX(minv_h)(&pc, F + (int64_t)s * N);
    }

    /* step 2: g_0 = r_0, g^_0 = M^{-1} r_0, w_0 = A g^_0, c_0 = q_1^H w_0,
     * e_0 = q_1^H r_0 */
    memcpy(G, r, (size_t)N * sizeof(S));
    if (pc_on)
        SFX(minv)(&pc, G, Gh);
    SFX(matvec)(N, rp, ci, av, Gh, W, ops);
    c[0] = SFX(dot)(N, Q, W, ops);
    if (c[0] == 0) {
        res->flag = -1;
        goto done;
    }
    e = SFX(dot)(N, Q, r, ops);

    for (j = 0;; ++j) {
        if (blk_ops && j < blk_cap)
            memcpy(blk_ops + 5 * j, ops, 5 * sizeof(int64_t));

        for (i = 1; i <= n - 1; ++i) {
            S *gi = G + (int64_t)i * N;   /* slot of g_{jn+i} */
            S *wi = W + (int64_t)i * N;   /* slot of w_{jn+i} (z_w) */

            /* steps 5-7 (x advances along g^) */
            alpha = e / c[i - 1];
            SFX(axpy)(N, alpha, Gh + (int64_t)(i - 1) * N, x, ops);
            SFX(axpy)(N, -alpha, W + (int64_t)(i - 1) * N, r, ops);
            err = SFX(nrm2)(N, r, ops) / bnrm2;
            iter++;
            RECORD();
            if (err < tol) {
                res->flag = 0;
                goto done;
            }
            if (iter >= maxit)
                goto done;

            /* step 8: e_{jn+i} = q_{i+1}^H r_{jn+i} */
            e = SFX(dot)(N, Q + (int64_t)i * N, r, ops);

            if (j >= 1) {
                /* steps 10-12: z_w = r + bt w_{(j-1)n+i}, g = bt g_{(j-1)n+i} */
                S bt = -e / c[i];
                SFX(xpay)(N, r, bt, wi, wi, ops);
                SFX(scal)(N, bt, gi, ops);
                /* steps 13-17: sweep the rest of block j-1 */
                for (int32_t s = i + 1; s <= n - 1; ++s) {
                    bt = -SFX(dot)(N, Q + (int64_t)s * N, wi, ops) / c[s];
                    SFX(axpy)(N, bt, W + (int64_t)s * N, wi, ops);
                    SFX(axpy)(N, bt, G + (int64_t)s * N, gi, ops);
                }
                /* step 18: g = z_w - g / omega_j */
                SFX(omega_corr)(N, wi, omega, gi, ops);
                /* steps 19-22: sweep block j with f_{s+1} */
                for (int32_t s = 0; s <= i - 1; ++s) {
                    S beta = -SFX(dot)(N, F + (int64_t)s * N, gi, ops) / c[s];
                    SFX(axpy)(N, beta, G + (int64_t)s * N, gi, ops);
                }
            } else {
                /* steps 24-29 (j = 0; omega is not used) */
                S beta = -SFX(dot)(N, F, r, ops) / c[0];
                SFX(xpay)(N, r, beta, G, gi, ops);
                for (int32_t s = 1; s <= i - 1; ++s) {
                    beta = -SFX(dot)(N, F + (int64_t)s * N, gi, ops) / c[s];
                    SFX(axpy)(N, beta, G + (int64_t)s * N, gi, ops);
                }
            }

            /* steps 31-32: g^ = M^{-1} g, w = A g^, c = q_{i+1}^H w */
            if (pc_on)
                SFX(minv)(&pc, gi, Gh + (int64_t)i * N);
            SFX(matvec)(N, rp, ci, av, Gh + (int64_t)i * N, wi, ops);
            c[i] = SFX(dot)(N, Q + (int64_t)i * N, wi, ops);
            if (c[i] == 0) {
                res->flag = -1;
                goto done;
            }
        }

        /* steps 34-36: alpha, x, u (u is kept in r) */
        i = n;
        alpha = e / c[n - 1];
        SFX(axpy)(N, alpha, Gh + (int64_t)(n - 1) * N, x, ops);
        SFX(axpy)(N, -alpha, W + (int64_t)(n - 1) * N, r, ops);
        err = SFX(nrm2)(N, r, ops) / bnrm2;
        if (err < tol) {
            iter++;
            RECORD();
            res->flag = 0;
            goto done;
        }

        /* step 37: u^ = M^{-1} u; step 38: omega = (A u^)^H u / ||A u^||^2 */
        if (pc_on)
            SFX(minv)(&pc, r, uh);
        SFX(matvec)(N, rp, ci, av, uh, z, ops);
        S zz = SFX(dot)(N, z, z, ops);
        if (zz == 0) {
            res->flag = -1;
            goto done;
        }
        S zu = SFX(dot)(N, z, r, ops);
        omega = zu / zz;
        /* Eq. 5.1: keep |rho| = |(Au)^H u| / (||Au|| ||u||) away from 0 */
        if (kappa > 0) {
            double nz = SFX(nrm2)(N, z, ops);
            double nu = SFX(nrm2)(N, r, ops);
            double arho = ABS(zu / (nz * nu));
            if (arho < kappa && arho != 0.0)
                omega = omega * kappa / arho;
        }
        if (omega == 0) {
            res->flag = -1;
            goto done;
        }

        /* steps 39-40: x += omega u^, r = u - omega A u^ */
        SFX(axpy)(N, omega, uh, x, ops);
        SFX(axpy)(N, -omega, z, r, ops);
        err = SFX(nrm2)(N, r, ops) / bnrm2;
        iter++;
        RECORD();
        if (err < tol) {
            res->flag = 0;
            goto done;
        }
        if (iter >= maxit)
            goto done;

        /* steps 41-44 */
        e = SFX(dot)(N, Q, r, ops);
        S bt = -e / c[0];
        SFX(xpay)(N, r, bt, W, W, ops);
        SFX(scal)(N, bt, G, ops);
        /* steps 45-49: sweep block j */
        for (int32_t s = 1; s <= n - 1; ++s) {
            bt = -SFX(dot)(N, Q + (int64_t)s * N, W, ops) / c[s];
            SFX(axpy)(N, bt, W + (int64_t)s * N, W, ops);
            SFX(axpy)(N, bt, G + (int64_t)s * N, G, ops);
        }
        /* step 50: g = z_w - g / omega_{j+1} */
        SFX(omega_corr)(N, W, omega, G, ops);
        /* step 50 (end): g^ = M^{-1} g; step 51: w = A g^, c = q_1^H w */
        if (pc_on)
            SFX(minv)(&pc, G, Gh);
        SFX(matvec)(N, rp, ci, av, Gh, W, ops);
        c[0] = SFX(dot)(N, Q, W, ops);
        if (c[0] == 0) {
            res->flag = -1;
            goto done;
        }
    }
#undef RECORD

done:
    res->iter = iter;
    res->err = err;
    res->j = (int32_t)j;
    res->i = i;
    free(G); free(W); free(F); free(r); free(z); free(c);
    if (pc_on) { free(Gh); free(uh); }
    return 0;
}
