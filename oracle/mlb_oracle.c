/*
 * CPU ORACLE for ML(n)BiCGStab (arXiv:1106.3678) — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential C in FP64 (double) and complex128 (double complex).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  The CUDA library never links, includes or calls anything
 * here, and nothing here comes from the CUDA library: the two share no code.
 *
 * What it computes, with the passage each part follows:
 *   orc_gn, orc_rn           index functions g_n(k) = floor((k-1)/n),
 *                            r_n(k) = k - n g_n(k)                  (§2, eq. 2.1)
 *   orc_spmv_{d,z}           y = A x, definition of the CSR product
 *   orc_ahq_{d,z}            F = A^H Q(:,1:n-1)            (Algorithm 4.1, step 2)
 *   orc_mlbicgstabt_{d,z}    ML(n)BiCGStabt = Algorithm 7.1 (M = I, which is
 *                            Algorithm 4.1, or a diagonal or ILU(0) M applied
 *                            as written), stopping rule and flags of §5, omega
 *                            guard of Eq. 5.1
 *   orc_ilu0_{d,z}           ILU(0) factors of A (the preconditioner of the
 *                            paper's experiments, §5; textbook definition)
 *   orc_minv_{d,z},          M^{-1} v and M^{-H} v for a diagonal or ILU(0) M
 *   orc_minv_h_{d,z}         (Algorithm 7.1, steps 2, 31, 37, 50)
 *   orc_qgauss               N(0,1) shadow vectors from the counter-based
 *                            generator the library documents: SplitMix64
 *                            (Steele, Lea & Flood, OOPSLA 2014) evaluated at
 *                            a counter, two uniforms -> Box–Muller (cosine
 *                            branch).  The paper fixes no generator.
 *
 * Parity pins (tests/test_oracle_*.py): Table 2.1 bit-exact; n = 1 against
 * an independently written textbook BiCGStab; n >= N finite termination and
 * block-0 bi-orthogonality (Algorithm 3.1 Petrov–Galerkin conditions);
 * agreement with a dense LU solve; Table 4.3 operation counts per block;
 * ILU(0): (L U)_ij = a_ij on A's pattern, exact LU when the pattern has no
 * fill, M^{-1} and M^{-H} against dense solves, one-step convergence when
 * M = A.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OP_MATVEC = 0, ORC_OP_DOT = 1, ORC_OP_SAXPY = 2, ORC_OP_SCALE = 3,
       ORC_OP_NORM = 4 };

typedef struct {
    int64_t iter;   /* k-steps performed */
    int32_t flag;   /* 0 converged, 1 iteration limit, -1 breakdown */
    int32_t j;      /* block index of the last step */
    int32_t i;      /* in-block index (1..n) of the last step */
    int32_t pad;
    double err;     /* last recursive relative residual */
    int64_t ops[5]; /* matvec, dot, saxpy, scale, norm counters */
} orc_result;

/* ---- §2: index functions ------------------------------------------------ */

/* g_n(k) = floor((k-1)/n), rounding toward minus infinity for every k. */
int64_t orc_gn(int64_t n, int64_t k)
{
    int64_t a = k - 1;
    int64_t q = a / n;           /* C division truncates toward zero */
    if ((a % n != 0) && ((a < 0) != (n < 0)))
        q -= 1;
    return q;
}

/* r_n(k) = k - n g_n(k), with range {1, ..., n}. */
int64_t orc_rn(int64_t n, int64_t k)
{
    return k - n * orc_gn(n, k);
}

/* ---- shadow-vector generator -------------------------------------------- */

/* Output number t (t = 0, 1, ...) of SplitMix64 seeded with `seed`: the
 * state after t+1 additions of the golden-ratio increment, then the
 * published finaliser. */
static uint64_t orc_splitmix64_at(uint64_t seed, uint64_t t)
{
    uint64_t z = seed + (t + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform on (0, 1]: the top 53 bits plus one, times 2^-53. */
static double orc_unit(uint64_t v)
{
    return ((double)(v >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* Normal number t: Box–Muller on outputs 2t and 2t+1 (cosine branch). */
double orc_normal_at(uint64_t seed, uint64_t t)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = orc_unit(orc_splitmix64_at(seed, 2u * t));
    double u2 = orc_unit(orc_splitmix64_at(seed, 2u * t + 1u));
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

/* Q (N x n, column-major, ld N): real entry e = col*N + row is normal
 * number e; a complex entry e takes normals 2e (real part) and 2e+1
 * (imaginary part), written interleaved (re, im). */
void orc_qgauss(uint64_t seed, int64_t N, int32_t n, int32_t is_complex,
                double *out)
{
    int64_t total = N * (int64_t)n;
    if (is_complex) {
        for (int64_t e = 0; e < total; ++e) {
            out[2 * e] = orc_normal_at(seed, (uint64_t)(2 * e));
            out[2 * e + 1] = orc_normal_at(seed, (uint64_t)(2 * e + 1));
        }
    } else {
        for (int64_t e = 0; e < total; ++e)
            out[e] = orc_normal_at(seed, (uint64_t)e);
    }
}

/* ---- multi-core build ----------------------------------------------------
 * Compiled a second time with ORC_PAR and OpenMP (liborc_par.so): the
 * same arithmetic, with elementwise loops shared among threads and inner
 * products and norms taken over fixed 1024-entry blocks, so its results
 * do not depend on the thread count (they differ from this sequential
 * build in rounding order only).  Used to time the oracle on all host
 * cores and to check long solves of large systems in reasonable time. */
#ifdef ORC_PAR
#include <omp.h>
void orc_par_set_threads(int32_t t) { omp_set_num_threads(t > 0 ? t : 1); }
int32_t orc_par_max_threads(void) { return (int32_t)omp_get_max_threads(); }
#endif

/* ---- the method, real FP64 ---------------------------------------------- */
#define S double
#define SFX(name) name##_d
#define CONJ(a) (a)
#define ABS2(a) ((a) * (a))
#define ABS(a) fabs(a)
#include "mlb_oracle_body.h"
#undef S
#undef SFX
#undef CONJ
#undef ABS2
#undef ABS

/* ---- the method, complex128 --------------------------------------------- */
#define S double complex
#define SFX(name) name##_z
#define CONJ(a) conj(a)
#define ABS2(a) (creal(a) * creal(a) + cimag(a) * cimag(a))
#define ABS(a) cabs(a)
#include "mlb_oracle_body.h"
#undef S
#undef SFX
#undef CONJ
#undef ABS2
#undef ABS
