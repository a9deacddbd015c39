/*
 * oracle.c -- plain, slow, FP64 CPU restatement of the randomized block BFGS
 * family of Gower & Richtarik, "Randomized Quasi-Newton Updates are Linearly
 * Convergent Matrix Inversion Algorithms" (arXiv:1602.01768).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library; the one thing both sides implement separately from its published
 * definition is the Philox4x32-10 counter-based generator used to draw the
 * sketches.
 *
 * Conventions.  Every matrix is column-major, FP64, with an explicit leading
 * dimension equal to its row count.  Products are plain loops (OpenMP over
 * output columns, which changes no arithmetic); no blocking, fusion or
 * reordering beyond what each equation states.  Equation names are the
 * paper's LaTeX labels.
 *
 * Pins (what each function is checked against, tests/test_oracle_*.py):
 *   philox          published known-answer vectors (tests/golden/philox_kat.txt)
 *   gauss sketch    moments of N(0,1); independence of columns/steps
 *   cholesky, gj    LAPACK (numpy) on random SPD matrices
 *   rbfgs step      sketch equation X+ A S = S, symmetry, positive
 *                   definiteness, error recursion, q=n one-step inverse,
 *                   fixed point, literal vs. expanded form, expected rate
 *   adarbfgs step   L+ L+^T equals the RBFGS iterate for S = L S~,
 *                   sketch equation, q=n one-step inverse, monotone F(A) error
 *   newton-schulz   textbook quadratic convergence to A^-1
 *   mr step         optimality of the step length along the MR direction
 *   residuals       exact vs. sampled estimator with all columns; closed forms
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads of the OpenMP loops (timing of the oracle on a chosen number of host cores). */
void orc_set_threads(int threads) { omp_set_num_threads(threads > 0 ? threads : 1); }

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 S-box built from two      */
/* 32x32->64 multiplies, with the key bumped by the Weyl constants between    */
/* rounds.                                                                    */
/* ------------------------------------------------------------------------- */
#define PHILOX_MUL0 0xD2511F53u
#define PHILOX_MUL1 0xCD9E8D57u
#define PHILOX_WEYL0 0x9E3779B9u
#define PHILOX_WEYL1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL0;
            k1 += PHILOX_WEYL1;
        }
        uint64_t p0 = (uint64_t)PHILOX_MUL0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter-word tags that keep the different draws of one (seed, stream, k)
 * apart.  Gaussian sketches use word 1 = column index (< 2^30). */
#define ORC_TAG_COORD 0xC0000000u /* coordinate-block / Floyd draws of a step */
#define ORC_TAG_COLS 0xD0000000u  /* residual column sample                 */

static void philox_at(uint64_t seed, uint32_t w0, uint32_t w1, uint64_t k, uint64_t stream,
                      uint32_t out[4])
{
    uint32_t ctr[4] = {w0, w1, (uint32_t)k, (uint32_t)stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* 24-bit uniform in (0,1): ((x >> 8) + 1/2) * 2^-24, exact in binary32 and binary64. */
static double u24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

static float f32_of_bits(uint32_t b)
{
    float f;
    memcpy(&f, &b, 4);
    return f;
}
static uint32_t bits_of_f32(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/*
 * The Gaussian sketch is defined through binary32 arithmetic in a fixed order
 * (each step one correctly rounded IEEE operation; polynomials by fmaf in
 * Horner order), so that any IEEE platform reproduces it bit for bit.  The
 * elementary functions are written out from their Taylor series:
 *
 * ln u for u in (0, 1): u = m 2^e with m in [sqrt(1/2), sqrt(2)) (exact),
 * ln m = 2 atanh(s), s = (m - 1) / (m + 1), |s| < 0.1716, and
 * atanh(s) = s + s^3/3 + s^5/5 + s^7/7 + s^9/9 (the next term is below
 * 2e-9 relative); ln u = e ln2_hi + (e ln2_lo + ln m) with ln2_hi holding 16
 * significant bits, so e ln2_hi is exact.
 */
#define ORC_LN2_HI 0.693145751953125f
#define ORC_LN2_LO 1.42860676e-06f

float orc_logf32(float u)
{
    uint32_t b = bits_of_f32(u);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = f32_of_bits((b & 0x007fffffu) | 0x3f800000u); /* [1, 2) */
    if (m > 1.41421354f) {
        m = m * 0.5f; /* exact */
        e += 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f); /* m - 1 exact (Sterbenz) */
    const float s2 = s * s;
    float p = fmaf(s2, 0.111111112f, 0.142857149f); /* 1/9, 1/7 */
    p = fmaf(s2, p, 0.200000003f);                  /* 1/5 */
    p = fmaf(s2, p, 0.333333343f);                  /* 1/3 */
    const float at = fmaf(s * s2, p, s);            /* atanh(s) */
    const float lm = 2.0f * at;                     /* exact */
    const float t = fmaf((float)e, ORC_LN2_LO, lm);
    return (float)e * ORC_LN2_HI + t;
}

/*
 * sin(pi x) and cos(pi x) for x in [0, 2]: k = nearest integer to 2x (2x is
 * exact), r = x - k/2 in [-1/4, 1/4] (exact), t = pi r (rounded), the Taylor
 * polynomials of sin t (to t^11) and cos t (to t^12), then the quarter turn
 * k mod 4 selects and signs them.
 */
#define ORC_PI_F 3.14159274f

void orc_sincospif32(float x, float *sp, float *cp)
{
    const float k = rintf(2.0f * x);
    const float r = x - 0.5f * k;
    const float t = r * ORC_PI_F;
    const float t2 = t * t;
    float ps = fmaf(t2, -2.50521079e-08f, 2.75573188e-06f); /* -1/11!, 1/9! */
    ps = fmaf(t2, ps, -1.98412701e-04f);                    /* -1/7! */
    ps = fmaf(t2, ps, 8.33333377e-03f);                     /* 1/5! */
    ps = fmaf(t2, ps, -0.166666672f);                       /* -1/3! */
    const float sn = fmaf(t * t2, ps, t);
    float pc = fmaf(t2, 2.08767570e-09f, -2.75573188e-07f); /* 1/12!, -1/10! */
    pc = fmaf(t2, pc, 2.48015876e-05f);                     /* 1/8! */
    pc = fmaf(t2, pc, -1.38888892e-03f);                    /* -1/6! */
    pc = fmaf(t2, pc, 4.16666679e-02f);                     /* 1/4! */
    pc = fmaf(t2, pc, -0.5f);                               /* -1/2! */
    const float cs = fmaf(t2, pc, 1.0f);
    switch ((int)k & 3) {
    case 0: *sp = sn; *cp = cs; break;
    case 1: *sp = cs; *cp = -sn; break;
    case 2: *sp = -sn; *cp = -cs; break;
    default: *sp = -cs; *cp = sn; break;
    }
}

/* Round a finite binary32 value to the nearest TF32 value (10 stored fraction
 * bits), ties to even. */
float orc_round_tf32(float z)
{
    uint32_t b = bits_of_f32(z);
    const uint32_t r = b & 0x1fffu;
    b &= ~0x1fffu;
    if (r > 0x1000u || (r == 0x1000u && (b & 0x2000u))) b += 0x2000u;
    return f32_of_bits(b);
}

/*
 * Gaussian sketch S~ (n x q) for step k.  The paper draws S~ with i.i.d.
 * standard normal entries (Sec. 9.3, AdaRBFGS_gauss; Sec. 10); it does not
 * fix a generator or a precision.  Reading used here: entries (4r+t, j),
 * t = 0..3, come from one Philox block with counter (r, j, k, stream) and key
 * (seed_lo, seed_hi), turned into normals by the Box-Muller transform on word
 * pairs (0,1), (2,3):
 *   rad = sqrt(-2 ln u_a),  z_a = rad cos(2 pi u_b),  z_b = rad sin(2 pi u_b),
 * evaluated in binary32 as above and rounded to the nearest TF32 value, so
 * every entry carries 11 significant bits and is exact in one tensor-core pass.
 */
void orc_gauss_sketch(uint64_t seed, uint64_t stream, uint64_t k, int n, int q, double *S)
{
    for (int j = 0; j < q; ++j) {
        for (int r = 0; 4 * r < n; ++r) {
            uint32_t w[4];
            philox_at(seed, (uint32_t)r, (uint32_t)j, k, stream, w);
            double z[4];
            for (int p = 0; p < 2; ++p) {
                /* binary32 uniforms: above 1/2 the 25-bit value rounds to even (1 is possible, giving 0) */
                const float ua = (float)u24(w[2 * p]), ub = (float)u24(w[2 * p + 1]);
                const float rad = sqrtf(-2.0f * orc_logf32(ua));
                float sn, cs;
                orc_sincospif32(2.0f * ub, &sn, &cs);
                z[2 * p] = orc_round_tf32(rad * cs);
                z[2 * p + 1] = orc_round_tf32(rad * sn);
            }
            for (int t = 0; t < 4 && 4 * r + t < n; ++t) S[(4 * r + t) + (size_t)j * n] = z[t];
        }
    }
}

/* floor(x * m / 2^32) for a 32-bit draw x: an unbiased-enough map to [0, m). */
static uint32_t scale32(uint32_t x, uint32_t m) { return (uint32_t)(((uint64_t)x * m) >> 32); }

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * m distinct indices of [0, n), uniformly (AdaRBFGS_cols, Sec. 10: "q distinct
 * coordinate vectors ... selected uniformly at random"; the paper gives no
 * procedure).  Reading: Floyd's algorithm -- for i = 0..m-1 with t = n-m+i,
 * draw d uniform in [0, t] from Philox (counter (i, tag, k, stream)), take d
 * unless already chosen, else take t -- then sort ascending.
 */
void orc_floyd_sample(uint64_t seed, uint64_t stream, uint64_t k, uint32_t tag, int n, int m,
                      int *out)
{
    for (int i = 0; i < m; ++i) {
        uint32_t t = (uint32_t)(n - m + i);
        uint32_t w[4];
        philox_at(seed, (uint32_t)i, tag, k, stream, w);
        int d = (int)scale32(w[0], t + 1u);
        int seen = 0;
        for (int a = 0; a < i; ++a)
            if (out[a] == d) seen = 1;
        out[i] = seen ? (int)t : d;
    }
    qsort(out, (size_t)m, sizeof(int), cmp_int);
}

/*
 * Trace-weighted coordinate block (RBFGS with the "convenient" probabilities
 * p_i = Tr(S_i^T A S_i) / Tr(S^T A S), Sec. 8.8 / Sec. 9.1, on the complete
 * discrete sampling formed by the fixed partition of [n] into contiguous
 * blocks C_b = [b q, min((b+1) q, n)), Def. 7.1).  With S_b = I_{:C_b} the
 * weight of block b is sum_{i in C_b} A_ii.  Reading (for bit-identical draws
 * on every implementation): w_b = max(1, floor(2^52 * s_b / T)) with
 * s_b summed in ascending i and T summed in ascending b, an exact integer
 * prefix sum, and one 64-bit draw r = w0 | w1 << 32 from counter
 * (0, ORC_TAG_COORD, k, stream) mapped to t = floor(r * W / 2^64); the block is
 * the b with P_b <= t < P_{b+1}.  Returns the block index; *first and *size
 * describe C_b.
 */
int orc_coord_trace_block(const double *A, int n, int q, uint64_t seed, uint64_t stream,
                          uint64_t k, int *first, int *size)
{
    int nb = (n + q - 1) / q;
    double *s = (double *)malloc(sizeof(double) * (size_t)nb);
    double T = 0.0;
    for (int b = 0; b < nb; ++b) {
        double acc = 0.0;
        for (int i = b * q; i < n && i < (b + 1) * q; ++i) acc += A[i + (size_t)i * n];
        s[b] = acc;
    }
    for (int b = 0; b < nb; ++b) T += s[b];
    uint64_t *P = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nb + 1));
    P[0] = 0;
    for (int b = 0; b < nb; ++b) {
        double wb = floor(ldexp(s[b] / T, 52));
        uint64_t w = (uint64_t)wb;
        if (w == 0) w = 1;
        P[b + 1] = P[b] + w;
    }
    uint32_t w[4];
    philox_at(seed, 0u, ORC_TAG_COORD, k, stream, w);
    uint64_t r = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    uint64_t t = (uint64_t)(((unsigned __int128)r * (unsigned __int128)P[nb]) >> 64);
    int b = 0;
    while (b + 1 < nb && P[b + 1] <= t) ++b;
    *first = b * q;
    *size = ((b + 1) * q <= n) ? q : n - b * q;
    free(s);
    free(P);
    return b;
}

/* ------------------------------------------------------------------------- */
/* Plain dense linear algebra (column-major).                                 */
/* ------------------------------------------------------------------------- */
#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* C (m x p) = A (m x kk) * B (kk x p) */
static void mm_nn(int m, int p, int kk, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < p; ++j) {
        double *c = C + IDX(0, j, m);
        for (int i = 0; i < m; ++i) c[i] = 0.0;
        for (int l = 0; l < kk; ++l) {
            double b = B[IDX(l, j, kk)];
            const double *a = A + IDX(0, l, m);
            for (int i = 0; i < m; ++i) c[i] += a[i] * b;
        }
    }
}

/* C (m x p) = A^T * B with A (kk x m), B (kk x p) */
static void mm_tn(int m, int p, int kk, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int l = 0; l < kk; ++l) acc += A[IDX(l, i, kk)] * B[IDX(l, j, kk)];
            C[IDX(i, j, m)] = acc;
        }
}

/* C (m x p) = A (m x kk) * B^T with B (p x kk) */
static void mm_nt(int m, int p, int kk, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < p; ++j) {
        double *c = C + IDX(0, j, m);
        for (int i = 0; i < m; ++i) c[i] = 0.0;
        for (int l = 0; l < kk; ++l) {
            double b = B[IDX(j, l, p)];
            const double *a = A + IDX(0, l, m);
            for (int i = 0; i < m; ++i) c[i] += a[i] * b;
        }
    }
}

/* Lower Cholesky M = C C^T, in place on the lower triangle (upper zeroed).
 * Returns 0, or -1 when a pivot is not positive and finite (M not SPD). */
int orc_cholesky(int q, double *M)
{
    for (int j = 0; j < q; ++j) {
        double d = M[IDX(j, j, q)];
        for (int l = 0; l < j; ++l) d -= M[IDX(j, l, q)] * M[IDX(j, l, q)];
        if (!(d > 0.0) || !isfinite(d)) return -1;
        double cjj = sqrt(d);
        M[IDX(j, j, q)] = cjj;
        for (int i = j + 1; i < q; ++i) {
            double v = M[IDX(i, j, q)];
            for (int l = 0; l < j; ++l) v -= M[IDX(i, l, q)] * M[IDX(j, l, q)];
            M[IDX(i, j, q)] = v / cjj;
        }
    }
    for (int j = 1; j < q; ++j)
        for (int i = 0; i < j; ++i) M[IDX(i, j, q)] = 0.0;
    return 0;
}

/* Solve C Y = B in place (C lower q x q, B q x p). */
static void trsm_lower(int q, int p, const double *C, double *B)
{
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < q; ++i) {
            double v = B[IDX(i, j, q)];
            for (int l = 0; l < i; ++l) v -= C[IDX(i, l, q)] * B[IDX(l, j, q)];
            B[IDX(i, j, q)] = v / C[IDX(i, i, q)];
        }
}

/* Solve C^T Y = B in place (C lower q x q, B q x p). */
static void trsm_lower_t(int q, int p, const double *C, double *B)
{
    for (int j = 0; j < p; ++j)
        for (int i = q - 1; i >= 0; --i) {
            double v = B[IDX(i, j, q)];
            for (int l = i + 1; l < q; ++l) v -= C[IDX(l, i, q)] * B[IDX(l, j, q)];
            B[IDX(i, j, q)] = v / C[IDX(i, i, q)];
        }
}

/* Gauss-Jordan inverse with partial pivoting (brute force for small n).
 * Returns 0 or -1 if A is singular to working precision. */
int orc_gauss_jordan(int n, const double *A, double *Ainv)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    memcpy(W, A, sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Ainv[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(W[IDX(i, c, n)]) > fabs(W[IDX(piv, c, n)])) piv = i;
        if (W[IDX(piv, c, n)] == 0.0) {
            free(W);
            return -1;
        }
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                double t = W[IDX(c, j, n)];
                W[IDX(c, j, n)] = W[IDX(piv, j, n)];
                W[IDX(piv, j, n)] = t;
                t = Ainv[IDX(c, j, n)];
                Ainv[IDX(c, j, n)] = Ainv[IDX(piv, j, n)];
                Ainv[IDX(piv, j, n)] = t;
            }
        double inv = 1.0 / W[IDX(c, c, n)];
        for (int j = 0; j < n; ++j) {
            W[IDX(c, j, n)] *= inv;
            Ainv[IDX(c, j, n)] *= inv;
        }
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            double f = W[IDX(i, c, n)];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                W[IDX(i, j, n)] -= f * W[IDX(c, j, n)];
                Ainv[IDX(i, j, n)] -= f * Ainv[IDX(c, j, n)];
            }
        }
    }
    free(W);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* RBFGS: Algorithm 3 with W = A^-1, i.e. the block BFGS update Eq. (qunac),  */
/* Sec. 8.8:                                                                  */
/*   X+ = S L S^T + (I - S L S^T A) X (I - A S L S^T),  L = (S^T A S)^-1.      */
/* ------------------------------------------------------------------------- */

/* Lambda = (S^T A S)^-1 from the lower Cholesky factor C of M = S^T A S. */
static void inverse_from_cholesky(int q, const double *C, double *Lam)
{
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) Lam[IDX(i, j, q)] = (i == j) ? 1.0 : 0.0;
    trsm_lower(q, q, C, Lam);
    trsm_lower_t(q, q, C, Lam);
}

/*
 * One RBFGS step with a given sketch S (n x q, full column rank), in place on
 * the symmetric iterate X.  form 0 evaluates Eq. (qunac) literally with
 * P = S Lambda S^T as an n x n matrix; form 1 evaluates the same update as
 * the symmetric rank-2q correction obtained by multiplying Eq. (qunac) out:
 *   G = A S, Y = X G, T = G^T Y,
 *   X+ = X + S Lambda S^T + S Lambda T Lambda S^T - S Lambda Y^T - Y Lambda S^T
 *      = X + S W^T + W S^T,   W = S (Lambda + Lambda T Lambda)/2 - Y Lambda.
 * Returns 0, or -1 when S^T A S is not positive definite.
 */
int orc_rbfgs_step(int n, const double *A, double *X, const double *S, int q, int form)
{
    size_t nq = (size_t)n * q, qq = (size_t)q * q, nn = (size_t)n * n;
    double *G = (double *)malloc(sizeof(double) * nq);
    double *M = (double *)malloc(sizeof(double) * qq);
    double *Lam = (double *)malloc(sizeof(double) * qq);
    int rc = 0;
    mm_nn(n, q, n, A, S, G);   /* G = A S     */
    mm_tn(q, q, n, S, G, M);   /* M = S^T A S */
    if (orc_cholesky(q, M) != 0) {
        rc = -1;
        goto out;
    }
    inverse_from_cholesky(q, M, Lam);
    if (form == 0) {
        double *SL = (double *)malloc(sizeof(double) * nq);
        double *P = (double *)malloc(sizeof(double) * nn);
        double *T1 = (double *)malloc(sizeof(double) * nn);
        double *T2 = (double *)malloc(sizeof(double) * nn);
        double *T3 = (double *)malloc(sizeof(double) * nn);
        mm_nn(n, q, q, S, Lam, SL); /* S Lambda        */
        mm_nt(n, n, q, SL, S, P);   /* P = S Lambda S^T */
        mm_nn(n, n, n, P, A, T1);   /* P A             */
        for (size_t e = 0; e < nn; ++e) T1[e] = -T1[e];
        for (int i = 0; i < n; ++i) T1[IDX(i, i, n)] += 1.0; /* I - P A */
        mm_nn(n, n, n, A, P, T2);   /* A P             */
        for (size_t e = 0; e < nn; ++e) T2[e] = -T2[e];
        for (int i = 0; i < n; ++i) T2[IDX(i, i, n)] += 1.0; /* I - A P */
        mm_nn(n, n, n, T1, X, T3);  /* (I - P A) X     */
        mm_nn(n, n, n, T3, T2, T1); /* ... (I - A P)   */
        for (size_t e = 0; e < nn; ++e) X[e] = P[e] + T1[e];
        free(SL); free(P); free(T1); free(T2); free(T3);
    } else {
        double *Y = (double *)malloc(sizeof(double) * nq);
        double *T = (double *)malloc(sizeof(double) * qq);
        double *TL = (double *)malloc(sizeof(double) * qq);
        double *B1 = (double *)malloc(sizeof(double) * qq);
        double *W = (double *)malloc(sizeof(double) * nq);
        double *YL = (double *)malloc(sizeof(double) * nq);
        mm_nn(n, q, n, X, G, Y);     /* Y = X G        */
        mm_tn(q, q, n, G, Y, T);     /* T = G^T X G    */
        mm_nn(q, q, q, T, Lam, TL);  /* T Lambda       */
        mm_nn(q, q, q, Lam, TL, B1); /* Lambda T Lambda */
        for (size_t e = 0; e < qq; ++e) B1[e] = 0.5 * (Lam[e] + B1[e]);
        mm_nn(n, q, q, S, B1, W);    /* S B1           */
        mm_nn(n, q, q, Y, Lam, YL);  /* Y Lambda       */
        for (size_t e = 0; e < nq; ++e) W[e] -= YL[e];
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int c = 0; c < q; ++c)
                    acc += S[IDX(i, c, n)] * W[IDX(j, c, n)] + W[IDX(i, c, n)] * S[IDX(j, c, n)];
                X[IDX(i, j, n)] += acc;
            }
        free(Y); free(T); free(TL); free(B1); free(W); free(YL);
    }
out:
    free(G); free(M); free(Lam);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* AdaRBFGS: Algorithm 4 with the factored update Eq. (Cholimprov), Sec. 9.3: */
/*   S = L S~,  L+ = L + S R ((S~^T S~)^{-1/2} S~^T - R^T S^T A L),            */
/* R any factor with R R^T = (S^T A S)^-1 and (S~^T S~)^{1/2} any factor G     */
/* with G G^T = S~^T S~.  Reading: lower Cholesky C C^T = S^T A S, D D^T =    */
/* S~^T S~, so R = C^{-T}, G = D, and                                         */
/*   L+ = L + S^ V,   S^ = S C^{-T},   V = D^{-1} S~^T - C^{-1} (A S)^T L.     */
/* (The line of Algorithm 4 that forms R from S~^T A S~ is read as S^T A S,   */
/* the definition of R in Eq. (Chol).)                                        */
/* ------------------------------------------------------------------------- */
int orc_adarbfgs_step(int n, const double *A, double *L, const double *St, int q)
{
    size_t nq = (size_t)n * q, qq = (size_t)q * q;
    double *S = (double *)malloc(sizeof(double) * nq);
    double *G = (double *)malloc(sizeof(double) * nq);
    double *C = (double *)malloc(sizeof(double) * qq);
    double *D = (double *)malloc(sizeof(double) * qq);
    double *W = (double *)malloc(sizeof(double) * nq); /* q x n */
    double *V = (double *)malloc(sizeof(double) * nq); /* q x n */
    double *Sh = (double *)malloc(sizeof(double) * nq);
    int rc = 0;
    mm_nn(n, q, n, L, St, S);  /* S = L S~        */
    mm_nn(n, q, n, A, S, G);   /* G = A S         */
    mm_tn(q, q, n, S, G, C);   /* C <- S^T A S    */
    if (orc_cholesky(q, C) != 0) {
        rc = -1;
        goto out;
    }
    mm_tn(q, q, n, St, St, D); /* D <- S~^T S~    */
    if (orc_cholesky(q, D) != 0) {
        rc = -2;
        goto out;
    }
    mm_tn(q, n, n, G, L, W);   /* W = (A S)^T L   */
    /* V = D^{-1} S~^T - C^{-1} W */
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < q; ++c) V[IDX(c, j, q)] = St[IDX(j, c, n)];
    trsm_lower(q, n, D, V);
    trsm_lower(q, n, C, W);
    for (size_t e = 0; e < nq; ++e) V[e] -= W[e];
    /* S^ = S C^{-T}: C S^^T = S^T, row by row */
    {
        double *row = (double *)malloc(sizeof(double) * (size_t)q);
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c < q; ++c) row[c] = S[IDX(i, c, n)];
            trsm_lower(q, 1, C, row);
            for (int c = 0; c < q; ++c) Sh[IDX(i, c, n)] = row[c];
        }
        free(row);
    }
    /* L += S^ V */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < q; ++c) {
            double v = V[IDX(c, j, q)];
            for (int i = 0; i < n; ++i) L[IDX(i, j, n)] += Sh[IDX(i, c, n)] * v;
        }
out:
    free(S); free(G); free(C); free(D); free(W); free(V); free(Sh);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Sketch drivers: draw S (or S~) for step k and apply the step.              */
/* kind 0: Gaussian (n x q); kind 1: trace-weighted coordinate block;          */
/* kind 2: q uniform distinct coordinates (Floyd).                             */
/* ------------------------------------------------------------------------- */
static int draw_sketch(int kind, const double *A, int n, int q, uint64_t seed, uint64_t stream,
                       uint64_t k, double *S, int *qk)
{
    if (kind == 0) {
        orc_gauss_sketch(seed, stream, k, n, q, S);
        *qk = q;
        return 0;
    }
    int *idx = (int *)malloc(sizeof(int) * (size_t)q);
    int m = q;
    if (kind == 1) {
        int first, size;
        orc_coord_trace_block(A, n, q, seed, stream, k, &first, &size);
        for (int t = 0; t < size; ++t) idx[t] = first + t;
        m = size;
    } else {
        orc_floyd_sample(seed, stream, k, ORC_TAG_COORD, n, q, idx);
    }
    memset(S, 0, sizeof(double) * (size_t)n * m);
    for (int t = 0; t < m; ++t) S[IDX(idx[t], t, n)] = 1.0;
    free(idx);
    *qk = m;
    return 0;
}

/* Run steps k0 .. k0+nsteps-1 of RBFGS.  Returns the number of steps done
 * (fewer than nsteps only on a Cholesky breakdown). */
int orc_rbfgs_run(int n, const double *A, double *X, int q, int kind, uint64_t seed,
                  uint64_t stream, uint64_t k0, int nsteps, int form)
{
    double *S = (double *)malloc(sizeof(double) * (size_t)n * q);
    int done = 0;
    for (int s = 0; s < nsteps; ++s) {
        int qk;
        draw_sketch(kind, A, n, q, seed, stream, k0 + (uint64_t)s, S, &qk);
        if (orc_rbfgs_step(n, A, X, S, qk, form) != 0) break;
        ++done;
    }
    free(S);
    return done;
}

/*
 * Approximate inverse preconditioning step, Eq. (BFGSas) of Sec. 8 (the
 * nonsymmetric row variant, Algorithm 1, with W = A^-1 for SPD A):
 *   X+ = X + S (S^T A S)^-1 S^T (I - A X),
 * computed as G = A S, Lambda = (S^T G)^-1 (Cholesky), X+ = X + S Lambda (S^T - G^T X)
 * (S^T A = G^T for symmetric A).  X need not be symmetric.  Returns -1
 * (X untouched) when S^T A S is not positive definite.
 */
int orc_aip_step(int n, const double *A, double *X, const double *S, int q)
{
    size_t nq = (size_t)n * q, qq = (size_t)q * q;
    double *G = (double *)malloc(sizeof(double) * nq);
    double *M = (double *)malloc(sizeof(double) * qq);
    double *Lam = (double *)malloc(sizeof(double) * qq);
    double *R = (double *)malloc(sizeof(double) * nq); /* q x n: S^T - G^T X */
    double *V = (double *)malloc(sizeof(double) * nq); /* q x n: Lambda R   */
    int rc = 0;
    mm_nn(n, q, n, A, S, G); /* G = A S     */
    mm_tn(q, q, n, S, G, M); /* M = S^T A S */
    if (orc_cholesky(q, M) != 0) {
        rc = -1;
        goto out;
    }
    inverse_from_cholesky(q, M, Lam);
    mm_tn(q, n, n, G, X, R); /* G^T X */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < q; ++c) R[IDX(c, j, q)] = S[IDX(j, c, n)] - R[IDX(c, j, q)];
    mm_nn(q, n, q, Lam, R, V);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int c = 0; c < q; ++c) acc += S[IDX(i, c, n)] * V[IDX(c, j, q)];
            X[IDX(i, j, n)] += acc;
        }
out:
    free(G); free(M); free(Lam); free(R); free(V);
    return rc;
}

/* Run steps k0 .. k0+nsteps-1 of the AIP update (kind 0 gauss, 1 coord trace). */
int orc_aip_run(int n, const double *A, double *X, int q, int kind, uint64_t seed, uint64_t stream,
                uint64_t k0, int nsteps)
{
    double *S = (double *)malloc(sizeof(double) * (size_t)n * q);
    int done = 0;
    for (int s = 0; s < nsteps; ++s) {
        int qk;
        draw_sketch(kind, A, n, q, seed, stream, k0 + (uint64_t)s, S, &qk);
        if (orc_aip_step(n, A, X, S, qk) != 0) break;
        ++done;
    }
    free(S);
    return done;
}

/* Run steps k0 .. k0+nsteps-1 of AdaRBFGS (kind 0 gauss, kind 2 cols). */
int orc_adarbfgs_run(int n, const double *A, double *L, int q, int kind, uint64_t seed,
                     uint64_t stream, uint64_t k0, int nsteps)
{
    double *St = (double *)malloc(sizeof(double) * (size_t)n * q);
    int done = 0;
    for (int s = 0; s < nsteps; ++s) {
        int qk;
        draw_sketch(kind, 0, n, q, seed, stream, k0 + (uint64_t)s, St, &qk);
        if (orc_adarbfgs_step(n, A, L, St, qk) != 0) break;
        ++done;
    }
    free(St);
    return done;
}

/* ------------------------------------------------------------------------- */
/* Comparison methods, Sec. 10.                                               */
/* ------------------------------------------------------------------------- */

/* Newton-Schulz, Eq. (Newton-Schulz): X+ = 2 X - X A X. */
void orc_ns_step(int n, const double *A, double *X)
{
    size_t nn = (size_t)n * n;
    double *AX = (double *)malloc(sizeof(double) * nn);
    double *XAX = (double *)malloc(sizeof(double) * nn);
    mm_nn(n, n, n, A, X, AX);
    mm_nn(n, n, n, X, AX, XAX);
    for (size_t e = 0; e < nn; ++e) X[e] = 2.0 * X[e] - XAX[e];
    free(AX);
    free(XAX);
}

/* Spectral-norm estimate by power iteration (stands in for MATLAB normest,
 * Sec. 10): v0 = 1/sqrt(n), v <- A v / ||A v||, iters times; returns ||A v||. */
double orc_power_norm(int n, const double *A, int iters)
{
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double sigma = 0.0;
    for (int i = 0; i < n; ++i) v[i] = 1.0 / sqrt((double)n);
    for (int it = 0; it < iters; ++it) {
        mm_nn(n, 1, n, A, v, w);
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += w[i] * w[i];
        sigma = sqrt(s);
        for (int i = 0; i < n; ++i) v[i] = w[i] / sigma;
    }
    free(v);
    free(w);
    return sigma;
}

/* Newton-Schulz start, Sec. 10: X0 = 0.99 A^T / sigma^2 (A symmetric). */
void orc_ns_init(int n, const double *A, double sigma, double *X)
{
    double s = 0.99 / (sigma * sigma);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) X[IDX(i, j, n)] = s * A[IDX(j, i, n)];
}

/* Minimal residual, Eq. (MRiter): R = I - A X,
 * X+ = X + [Tr(R^T A X R) / Tr((A X R)^T A X R)] X R.  Returns the step length. */
double orc_mr_step(int n, const double *A, double *X)
{
    size_t nn = (size_t)n * n;
    double *R = (double *)malloc(sizeof(double) * nn);
    double *XR = (double *)malloc(sizeof(double) * nn);
    double *AXR = (double *)malloc(sizeof(double) * nn);
    mm_nn(n, n, n, A, X, R);
    for (size_t e = 0; e < nn; ++e) R[e] = -R[e];
    for (int i = 0; i < n; ++i) R[IDX(i, i, n)] += 1.0;
    mm_nn(n, n, n, X, R, XR);
    mm_nn(n, n, n, A, XR, AXR);
    double num = 0.0, den = 0.0;
    for (size_t e = 0; e < nn; ++e) {
        num += R[e] * AXR[e];
        den += AXR[e] * AXR[e];
    }
    double alpha = (den > 0.0) ? num / den : 0.0;
    for (size_t e = 0; e < nn; ++e) X[e] += alpha * XR[e];
    free(R); free(XR); free(AXR);
    return alpha;
}

/* MR start, Sec. 10: X0 = (Tr A / Tr(A A^T)) I. */
void orc_mr_init(int n, const double *A, double *X)
{
    double tr = 0.0, tr2 = 0.0;
    for (int i = 0; i < n; ++i) tr += A[IDX(i, i, n)];
    for (size_t e = 0; e < (size_t)n * n; ++e) tr2 += A[e] * A[e];
    for (size_t e = 0; e < (size_t)n * n; ++e) X[e] = 0.0;
    for (int i = 0; i < n; ++i) X[IDX(i, i, n)] = tr / tr2;
}

/* ------------------------------------------------------------------------- */
/* Residual monitor: ||I - X A||_F / sqrt(n) (equal to ||I - A X||_F/sqrt(n)  */
/* for symmetric X and A), the stopping quantity of Sec. 10 without its       */
/* normalisation by ||I - A X0||_F.                                           */
/* ------------------------------------------------------------------------- */
double orc_residual(int n, const double *A, const double *X)
{
    size_t nn = (size_t)n * n;
    double *XA = (double *)malloc(sizeof(double) * nn);
    mm_nn(n, n, n, X, A, XA);
    double acc = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double e = ((i == j) ? 1.0 : 0.0) - XA[IDX(i, j, n)];
            acc += e * e;
        }
    free(XA);
    return sqrt(acc / n);
}

/* Same for the factored iterate X = L L^T (Eq. X_k = L_k L_k^T, Sec. 9.2). */
double orc_residual_factored(int n, const double *A, const double *L)
{
    size_t nn = (size_t)n * n;
    double *X = (double *)malloc(sizeof(double) * nn);
    mm_nt(n, n, n, L, L, X);
    double r = orc_residual(n, A, X);
    free(X);
    return r;
}

/*
 * Column-sampled estimate: J = m distinct columns (Floyd, counter tag
 * ORC_TAG_COLS, key = col_seed, k = stream = 0), and
 *   est = sqrt( (1/m) sum_{j in J} || e_j - X A e_j ||^2 ),
 * which is unbiased for ||I - X A||_F^2 / n and exact when m = n.  When L is
 * non-null, X = L L^T is applied as L (L^T (A e_j)).
 */
double orc_residual_sampled(int n, const double *A, const double *X, const double *L, int m,
                            uint64_t col_seed)
{
    int *J = (int *)malloc(sizeof(int) * (size_t)m);
    orc_floyd_sample(col_seed, 0, 0, ORC_TAG_COLS, n, m, J);
    /* the m columns A e_j side by side, so each product below is one call whose
     * OpenMP loop runs over the m columns (every column's sums in the same order
     * as a one-column product) */
    double *AE = (double *)malloc(sizeof(double) * (size_t)n * m);
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * m);
    for (int t = 0; t < m; ++t) memcpy(AE + IDX(0, t, n), A + IDX(0, J[t], n), sizeof(double) * (size_t)n);
    if (L) {
        double *Y = (double *)malloc(sizeof(double) * (size_t)n * m);
        mm_tn(n, m, n, L, AE, Y); /* L^T A e_J     */
        mm_nn(n, m, n, L, Y, Z);  /* L L^T A e_J   */
        free(Y);
    } else {
        mm_nn(n, m, n, X, AE, Z); /* X A e_J       */
    }
    double acc = 0.0;
    for (int t = 0; t < m; ++t) {
        const int j = J[t];
        for (int i = 0; i < n; ++i) {
            double e = ((i == j) ? 1.0 : 0.0) - Z[IDX(i, t, n)];
            acc += e * e;
        }
    }
    free(J);
    free(AE);
    free(Z);
    return sqrt(acc / m);
}
