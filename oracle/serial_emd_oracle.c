/*
 * Serial-EMD oracle: a plain, slow, FP64 CPU statement of the Serial-EMD method
 * (Zhang et al., "Serial-EMD: Fast Empirical Mode Decomposition Method for
 * Multi-dimensional Signals Based on Serialization", arXiv 2106.15319).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file. The CUDA library does not
 * link it, call it, or share any code, header or table with it.
 *
 * Every step follows the paper in its order and notation:
 *   serialization ........ Sec. 3.2 (vector a, sub-matrices X_A / X_B, matrix E,
 *                          matrix T, t = vec(T), x = t_{1:(M+D)N-D})
 *   1D EMD ............... Sec. 2.1, Eq. (1) and sifting Steps 1-5
 *   EEMD ................. Sec. 2.2, Steps 1-3
 *   CEEMDAN .............. Sec. 2.2, the second list of Steps 1-4
 *   de-serialization ..... Sec. 3.3 (pad R with Z, reshape, drop the last D rows)
 * Where the paper is silent (interpolant, stop rule, end effects, ties) the
 * readings are fixed in one place each and named "Reading n" below:
 *   Reading 1  transition indices (0-based) of Sec. 3.2:
 *              x[i(M+D)+M+r] = (r+1)/(D+1) * X[D-1-r, i+1] + (D-r)/(D+1) * X[M-1-r, i]
 *   Reading 5  extremum rule: maximum at k iff h[k-1] < h[k] >= h[k+1],
 *              minimum at k iff h[k-1] > h[k] <= h[k+1], 1 <= k <= L-2;
 *              the two end samples are never extrema.
 *   Reading 6  envelopes are natural cubic splines with knots at the integer
 *              sample indices of the extrema (Sec. 1 names the cubic spline of
 *              standard EMD).
 *   Reading 6b not-a-knot ends (a plan option; Sec. 1 names the cubic spline
 *              without its end conditions): the third derivative is continuous
 *              at the second and the second-to-last knot, so the first two and
 *              the last two intervals each carry one cubic. Knot sequences with
 *              fewer than four knots keep the natural ends. Selected by adding
 *              OR_SPLINE_NOT_A_KNOT to the boundary code.
 *   Reading 7  mirror boundary: the first p = min(P, n) knots are reflected to
 *              -t_j and the last p to 2(L-1) - t_j, with the same values.
 *              ENDPOINTS alternative: (0, h[0]) and (L-1, h[L-1]) become knots.
 *   Reading 8  SD stop: SD = sum (h_prev - h)^2 / sum h_prev^2 < threshold,
 *              tested after each sift, at most max_sifts sifts.
 *   Reading 8b S-number stop (a plan option; the paper names no rule): after each
 *              sift, count the sifted signal's extrema (maxima + minima, Reading 5)
 *              and zero crossings (pairs k, k+1 where exactly one of the two samples
 *              is negative); sifting stops once S consecutive sifts have each left
 *              counts that differ by at most one, or after max_sifts sifts. S is
 *              passed in fixed_sifts under this rule.
 *   Reading 9  an IMF is started only if n_max >= 1, n_min >= 1 and
 *              n_max + n_min >= 3; otherwise the decomposition ends and the
 *              remainder is the residue. The same test on the sifted signal
 *              mid-sift stops the sifting and commits the signal as the IMF.
 *   Reading 11 EEMD noise is added to the serialized signal; beta is
 *              noise_rel_std times the population std of x; trials with fewer
 *              IMFs contribute zeros to the average.
 *   Reading 11b white noise drawn by the library itself (when the caller passes no
 *              noise): realization m, serialized sample p takes 32-bit word p mod 4
 *              of the Philox4x32-10 block with counter (p div 4, m, 0, 0) and key
 *              (seed low word, seed high word) (Salmon, Moraes, Dror and Shaw,
 *              "Parallel random numbers: as easy as 1, 2, 3", SC 2011); the word u
 *              gives the odd integer i = 2 (u >> 9) - (2^23 - 1) and the sample
 *              w = i * (sqrt(3) / 2^23) in FP64, uniform on (-sqrt 3, sqrt 3): zero
 *              mean, unit variance, independent samples (white). The paper asks for
 *              white noise of a given deviation without naming its distribution.
 *   Reading 12 CEEMDAN (Sec. 2.2, Steps 1-4): E_k(w) is the k-th EMD mode of the
 *              noise realization w (zero past its IMF count). Stage k = 0, 1, ...
 *              starts from the residue r_k (r_0 = x) and runs only if r_k passes
 *              Reading 9; beta_k is noise_rel_std times the population std of
 *              r_k. Mode k+1 is the trial average of the first EMD mode of
 *              r_k + beta_k w^(m) for k = 0 (the first EEMD mode, Step 1) and of
 *              r_k + beta_k E_k(w^(m)) for k >= 1 (Steps 2 and 4; Step 4's
 *              "c_2" is read as the mode being built); r_{k+1} = r_k - mode
 *              (Step 3). Trials whose input has no IMF contribute zeros.
 *
 * store_f32 (off for the reference decomposition): rounds the sifted signal to
 * single precision at IMF start and after every sift, the two points where the
 * FP32 form of the method stores it. All arithmetic stays FP64. Running the
 * oracle both ways measures how far single-precision storage alone moves each
 * IMF, which bounds what any FP32-storage implementation can match.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_STOP_FIXED 0
#define OR_STOP_SD 1
#define OR_STOP_SNUMBER 2
#define OR_BOUNDARY_MIRROR 0
#define OR_BOUNDARY_ENDPOINTS 1
#define OR_SPLINE_NOT_A_KNOT 16 /* flag added to the boundary code, Reading 6b */

/* ---------------------------------------------------------------- Sec. 3.2 */

/* Length of the serialized signal, Sec. 3.2: x has MN + DN - D samples. */
int64_t oracle_serial_length(int64_t M, int64_t N, int64_t D)
{
    return M * N + D * N - D;
}

/*
 * Sec. 3.2. X holds N signals of length M, signal i at X[i*M .. i*M+M-1]
 * (the columns x_i of the paper's M x N matrix). T = [X ; E z] is (M+D) x N,
 * t = vec(T) stacks its columns, and x drops the trailing zero vector z.
 * E = X_A^f (.) a u^T + X_B^f (.) a^f u^T with a_r = r/(D+1) (1-based r),
 * X_A = X_{1:D, 2:N}, X_B = X_{M-D+1:M, 1:N-1}; f flips the first dimension.
 */
void oracle_serialize(const double *X, int64_t M, int64_t N, int64_t D, double *x)
{
    int64_t i, m, r;
    for (i = 0; i < N; ++i) {
        /* column i of T: first the M samples of signal i */
        for (m = 0; m < M; ++m)
            x[i * (M + D) + m] = X[i * M + m];
        if (i == N - 1)
            break; /* the last column of T ends in z, which x drops */
        /* then the D transition samples E[:, i] (0-based r) */
        for (r = 0; r < D; ++r) {
            double a_r = (double)(r + 1) / (double)(D + 1);  /* a     */
            double af_r = (double)(D - r) / (double)(D + 1); /* a^f   */
            double xa_f = X[(i + 1) * M + (D - 1 - r)];      /* X_A^f */
            double xb_f = X[i * M + (M - 1 - r)];            /* X_B^f */
            x[i * (M + D) + M + r] = xa_f * a_r + xb_f * af_r;
        }
    }
}

/*
 * Sec. 3.3. R is K x L (IMF-major, L = MN + DN - D). T = [R ; Z] is padded with
 * D zeros, reshaped to (M+D) x N x K and the last D rows dropped, leaving
 * IMF (M x N x K). Output layout: IMF[k*N*M + i*M + m].
 */
void oracle_deserialize(const double *R, int64_t K, int64_t M, int64_t N, int64_t D,
                        double *IMF)
{
    int64_t L = oracle_serial_length(M, N, D), k, i, m;
    for (k = 0; k < K; ++k)
        for (i = 0; i < N; ++i)
            for (m = 0; m < M; ++m)
                IMF[k * N * M + i * M + m] = R[k * L + i * (M + D) + m];
}

/* ------------------------------------------------------ Sec. 2.1, Step 1 */

/* Reading 5. Writes ascending indices; returns counts through n_max / n_min. */
void oracle_extrema(const double *h, int64_t L, int32_t *t_max, int64_t *n_max,
                    int32_t *t_min, int64_t *n_min)
{
    int64_t k, a = 0, b = 0;
    for (k = 1; k + 1 < L; ++k) {
        if (h[k - 1] < h[k] && h[k] >= h[k + 1])
            t_max[a++] = (int32_t)k;
        if (h[k - 1] > h[k] && h[k] <= h[k + 1])
            t_min[b++] = (int32_t)k;
    }
    *n_max = a;
    *n_min = b;
}

/* ------------------------------------------------------ Sec. 2.1, Step 2 */

/*
 * Natural cubic spline through (s_j, v_j), j = 0..n-1, s strictly increasing,
 * n >= 2 (Reading 6). Second derivatives Mj satisfy M_0 = M_{n-1} = 0 and, for
 * 0 < j < n-1,
 *   h_{j-1} M_{j-1} + 2 (h_{j-1} + h_j) M_j + h_j M_{j+1}
 *       = 6 [ (v_{j+1} - v_j)/h_j - (v_j - v_{j-1})/h_{j-1} ],  h_j = s_{j+1} - s_j.
 * Solved by the Thomas algorithm (forward elimination, back substitution).
 */
void oracle_spline_second_derivs(const double *s, const double *v, int64_t n, double *Mj)
{
    int64_t j, m = n - 2; /* interior unknowns j = 1..n-2 */
    double *cp, *dp;
    Mj[0] = 0.0;
    Mj[n - 1] = 0.0;
    if (m <= 0)
        return;
    cp = (double *)malloc((size_t)m * sizeof(double));
    dp = (double *)malloc((size_t)m * sizeof(double));
    for (j = 1; j <= n - 2; ++j) {
        double hl = s[j] - s[j - 1], hr = s[j + 1] - s[j];
        double a = hl, b = 2.0 * (hl + hr), c = hr;
        double d = 6.0 * ((v[j + 1] - v[j]) / hr - (v[j] - v[j - 1]) / hl);
        int64_t q = j - 1;
        if (q == 0) {
            cp[q] = c / b;
            dp[q] = d / b;
        } else {
            double den = b - a * cp[q - 1];
            cp[q] = c / den;
            dp[q] = (d - a * dp[q - 1]) / den;
        }
    }
    Mj[n - 2] = dp[m - 1];
    for (j = n - 3; j >= 1; --j)
        Mj[j] = dp[j - 1] - cp[j - 1] * Mj[j + 1];
    free(cp);
    free(dp);
}

/*
 * Not-a-knot spline (Reading 6b): the same interior rows, with the two end conditions
 *   (M_1 - M_0) / h_0 = (M_2 - M_1) / h_1 and
 *   (M_{n-1} - M_{n-2}) / h_{n-2} = (M_{n-2} - M_{n-3}) / h_{n-3}.
 * They give M_0 = ((h_0 + h_1) M_1 - h_0 M_2) / h_1 and the mirror image for M_{n-1};
 * substituted into rows 1 and n-2 they leave a tridiagonal system in M_1..M_{n-2}
 * (Thomas algorithm), after which M_0 and M_{n-1} follow. n < 4: natural ends.
 */
void oracle_spline_second_derivs_nak(const double *s, const double *v, int64_t n, double *Mj)
{
    int64_t j, m = n - 2;
    double *cp, *dp;
    if (n < 4) {
        oracle_spline_second_derivs(s, v, n, Mj);
        return;
    }
    cp = (double *)malloc((size_t)m * sizeof(double));
    dp = (double *)malloc((size_t)m * sizeof(double));
    for (j = 1; j <= n - 2; ++j) {
        double hl = s[j] - s[j - 1], hr = s[j + 1] - s[j];
        double a = hl, b = 2.0 * (hl + hr), c = hr;
        double d = 6.0 * ((v[j + 1] - v[j]) / hr - (v[j] - v[j - 1]) / hl);
        int64_t q = j - 1;
        if (j == 1) { /* M_0 substituted */
            b = b + hl * (hl + hr) / hr;
            c = hr - hl * hl / hr;
            a = 0.0;
        }
        if (j == n - 2) { /* M_{n-1} substituted */
            b = b + hr * (hl + hr) / hl;
            a = hl - hr * hr / hl;
            c = 0.0;
        }
        if (q == 0) {
            cp[q] = c / b;
            dp[q] = d / b;
        } else {
            double den = b - a * cp[q - 1];
            cp[q] = c / den;
            dp[q] = (d - a * dp[q - 1]) / den;
        }
    }
    Mj[n - 2] = dp[m - 1];
    for (j = n - 3; j >= 1; --j)
        Mj[j] = dp[j - 1] - cp[j - 1] * Mj[j + 1];
    {
        double h0 = s[1] - s[0], h1 = s[2] - s[1];
        double ha = s[n - 2] - s[n - 3], hb = s[n - 1] - s[n - 2];
        Mj[0] = ((h0 + h1) * Mj[1] - h0 * Mj[2]) / h1;
        Mj[n - 1] = ((ha + hb) * Mj[n - 2] - hb * Mj[n - 3]) / ha;
    }
    free(cp);
    free(dp);
}

/* Value of the natural cubic spline at abscissa u, with s_j <= u <= s_{j+1}. */
static double spline_eval_interval(const double *s, const double *v, const double *Mj,
                                   int64_t j, double u)
{
    double h = s[j + 1] - s[j];
    double A = (s[j + 1] - u) / h, B = (u - s[j]) / h;
    return A * v[j] + B * v[j + 1] +
           ((A * A * A - A) * Mj[j] + (B * B * B - B) * Mj[j + 1]) * (h * h) / 6.0;
}

/*
 * Envelope through the knots t (n >= 1 extrema of one kind) of a signal of
 * length L, evaluated at k = 0..L-1 (Sec. 2.1 Step 2 with Readings 6 and 7).
 * h is the signal (needed for the ENDPOINTS rule only).
 */
void oracle_envelope(const double *h, int64_t L, const int32_t *t, int64_t n,
                     int boundary, int mirror_knots, double *env)
{
    const int nak = (boundary & OR_SPLINE_NOT_A_KNOT) != 0;
    int64_t p, nk, j, k, q = 0;
    boundary &= ~OR_SPLINE_NOT_A_KNOT;
    p = (boundary == OR_BOUNDARY_MIRROR) ? (n < mirror_knots ? n : mirror_knots) : 0;
    nk = (boundary == OR_BOUNDARY_MIRROR) ? n + 2 * p : n + 2;
    double *s = (double *)malloc((size_t)nk * sizeof(double));
    double *v = (double *)malloc((size_t)nk * sizeof(double));
    double *Mj = (double *)malloc((size_t)nk * sizeof(double));
    if (boundary == OR_BOUNDARY_MIRROR) {
        for (j = p - 1; j >= 0; --j) { /* left mirror: -t_{p-1} < ... < -t_0 */
            s[q] = -(double)t[j];
            v[q++] = h[t[j]];
        }
        for (j = 0; j < n; ++j) {
            s[q] = (double)t[j];
            v[q++] = h[t[j]];
        }
        for (j = n - 1; j >= n - p; --j) { /* right mirror: 2(L-1) - t_{n-1} < ... */
            s[q] = 2.0 * (double)(L - 1) - (double)t[j];
            v[q++] = h[t[j]];
        }
    } else {
        s[q] = 0.0;
        v[q++] = h[0];
        for (j = 0; j < n; ++j) {
            s[q] = (double)t[j];
            v[q++] = h[t[j]];
        }
        s[q] = (double)(L - 1);
        v[q++] = h[L - 1];
    }
    if (nak)
        oracle_spline_second_derivs_nak(s, v, nk, Mj);
    else
        oracle_spline_second_derivs(s, v, nk, Mj);
    j = 0;
    for (k = 0; k < L; ++k) {
        while (j + 2 < nk && s[j + 1] <= (double)k)
            ++j;
        env[k] = spline_eval_interval(s, v, Mj, j, (double)k);
    }
    free(s);
    free(v);
    free(Mj);
}

/* ---------------------------------------------------- Sec. 2.1, Steps 1-4 */

/*
 * One sift: extrema of h, the two envelopes, their mean m, and h_out = h - m.
 * Returns 0 and writes sum (h - h_out)^2 and sum h^2 through sd_num / sd_den,
 * or returns 1 (h_out untouched) when either kind of extremum is missing.
 */
int oracle_sift(const double *h, int64_t L, int boundary, int mirror_knots,
                double *h_out, double *sd_num, double *sd_den)
{
    int32_t *tmax = (int32_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int32_t));
    int32_t *tmin = (int32_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int32_t));
    double *emax = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
    double *emin = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
    int64_t nmax, nmin, k;
    double num = 0.0, den = 0.0;
    int rc = 0;
    oracle_extrema(h, L, tmax, &nmax, tmin, &nmin);                 /* Step 1 */
    if (nmax < 1 || nmin < 1) {
        rc = 1;
        goto out;
    }
    oracle_envelope(h, L, tmax, nmax, boundary, mirror_knots, emax); /* Step 2 */
    oracle_envelope(h, L, tmin, nmin, boundary, mirror_knots, emin);
    for (k = 0; k < L; ++k) {
        double m = (emin[k] + emax[k]) / 2.0;                        /* Step 3 */
        double s = h[k] - m;                                         /* Step 4 */
        num += (h[k] - s) * (h[k] - s);
        den += h[k] * h[k];
        h_out[k] = s;
    }
    *sd_num = num;
    *sd_den = den;
out:
    free(tmax);
    free(tmin);
    free(emax);
    free(emin);
    return rc;
}

/* Reading 8b: zero crossings of h, pairs (k, k+1) with exactly one negative sample. */
int64_t oracle_zero_crossings(const double *h, int64_t L)
{
    int64_t k, n = 0;
    for (k = 0; k + 1 < L; ++k)
        if ((h[k] < 0.0) != (h[k + 1] < 0.0))
            ++n;
    return n;
}

/* Reading 9: may an IMF be started from (or sifting continue on) h? */
static int has_enough_extrema(const double *h, int64_t L, int32_t *scratch_a,
                              int32_t *scratch_b)
{
    int64_t nmax, nmin;
    oracle_extrema(h, L, scratch_a, &nmax, scratch_b, &nmin);
    return nmax >= 1 && nmin >= 1 && nmax + nmin >= 3;
}

/* ------------------------------------------------ Sec. 2.1, Eq. (1), Step 5 */

/*
 * Standard 1D EMD of x (length L): x = sum_i c_i + r (Eq. 1). imfs is K x L
 * (slots past the produced count are zero-filled), residue is L. The stop rule
 * is a fixed sift count (stop = OR_STOP_FIXED, fixed_sifts), the SD rule of
 * Reading 8 or the S-number rule of Reading 8b (S in fixed_sifts). sifts_per_imf
 * (length K, may be NULL) receives each IMF's sift count. store_f32: see the
 * header. Returns the number of IMFs produced.
 */
static void round_to_single(double *h, int64_t L)
{
    int64_t k;
    for (k = 0; k < L; ++k)
        h[k] = (double)(float)h[k];
}

int oracle_emd(const double *x, int64_t L, int K, int stop, int fixed_sifts,
               double sd_threshold, int max_sifts, int boundary, int mirror_knots,
               double *imfs, double *residue, int *sifts_per_imf, int store_f32)
{
    double *r = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
    double *h = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
    double *hn = (double *)malloc((size_t)(L > 0 ? L : 1) * sizeof(double));
    int32_t *sa = (int32_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int32_t));
    int32_t *sb = (int32_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int32_t));
    int i = 0, k;
    int64_t q;
    memcpy(r, x, (size_t)L * sizeof(double));
    memset(imfs, 0, (size_t)K * (size_t)L * sizeof(double));
    if (sifts_per_imf)
        for (k = 0; k < K; ++k)
            sifts_per_imf[k] = 0;
    for (i = 0; i < K; ++i) {
        int sifts = 0, scount = 0;
        if (!has_enough_extrema(r, L, sa, sb))
            break; /* Reading 9: r is the residue */
        memcpy(h, r, (size_t)L * sizeof(double));
        if (store_f32)
            round_to_single(h, L);
        for (;;) {
            double num, den, *tmp;
            if (stop == OR_STOP_FIXED && sifts >= fixed_sifts)
                break;
            if (!has_enough_extrema(h, L, sa, sb))
                break; /* Reading 9 mid-sift: commit h */
            if (oracle_sift(h, L, boundary, mirror_knots, hn, &num, &den) != 0)
                break;
            ++sifts;
            tmp = h;
            h = hn;
            hn = tmp;
            if (store_f32)
                round_to_single(h, L);
            if (stop == OR_STOP_SD) {
                if (num / den < sd_threshold || sifts >= max_sifts)
                    break; /* Reading 8 */
            } else if (stop == OR_STOP_SNUMBER) {
                int64_t nmax, nmin, d;
                oracle_extrema(h, L, sa, &nmax, sb, &nmin);
                d = nmax + nmin - oracle_zero_crossings(h, L);
                scount = (d >= -1 && d <= 1) ? scount + 1 : 0;
                if (scount >= fixed_sifts || sifts >= max_sifts)
                    break; /* Reading 8b */
            }
        }
        /* Step 5: c_i = h, and the next IMF is sifted from r - c_i */
        for (q = 0; q < L; ++q) {
            imfs[(int64_t)i * L + q] = h[q];
            r[q] = r[q] - h[q];
        }
        if (sifts_per_imf)
            sifts_per_imf[i] = sifts;
    }
    memcpy(residue, r, (size_t)L * sizeof(double));
    free(r);
    free(h);
    free(hn);
    free(sa);
    free(sb);
    return i;
}

/* ------------------------------------------------------- Sec. 2.2, EEMD */

/* Population standard deviation of x (Reading 11 sets beta from it). */
double oracle_std(const double *x, int64_t L)
{
    double mean = 0.0, var = 0.0;
    int64_t k;
    for (k = 0; k < L; ++k)
        mean += x[k];
    mean /= (double)L;
    for (k = 0; k < L; ++k)
        var += (x[k] - mean) * (x[k] - mean);
    return sqrt(var / (double)L);
}

/*
 * EEMD (Sec. 2.2): x^(m) = x + beta w^(m) for m = 1..trials (w given, trials x L,
 * row m is one white-noise realization), each decomposed by EMD; the i-th mode
 * of x is the average of the i-th modes (zeros where a trial has fewer IMFs).
 * The residue is averaged the same way. Returns the largest IMF count.
 */
int oracle_eemd(const double *x, int64_t L, const double *w, int trials, double beta,
                int K, int stop, int fixed_sifts, double sd_threshold, int max_sifts,
                int boundary, int mirror_knots, double *imfs, double *residue, int store_f32)
{
    double *xm = (double *)malloc((size_t)L * sizeof(double));
    double *cm = (double *)malloc((size_t)K * (size_t)L * sizeof(double));
    double *rm = (double *)malloc((size_t)L * sizeof(double));
    int m, nmax = 0;
    int64_t q;
    memset(imfs, 0, (size_t)K * (size_t)L * sizeof(double));
    memset(residue, 0, (size_t)L * sizeof(double));
    for (m = 0; m < trials; ++m) {
        int n;
        for (q = 0; q < L; ++q)
            xm[q] = x[q] + beta * w[(int64_t)m * L + q]; /* Step 1 */
        n = oracle_emd(xm, L, K, stop, fixed_sifts, sd_threshold, max_sifts, boundary,
                       mirror_knots, cm, rm, NULL, store_f32); /* Step 2 */
        if (n > nmax)
            nmax = n;
        for (q = 0; q < (int64_t)K * L; ++q)
            imfs[q] += cm[q];
        for (q = 0; q < L; ++q)
            residue[q] += rm[q];
    }
    for (q = 0; q < (int64_t)K * L; ++q) /* Step 3 */
        imfs[q] /= (double)trials;
    for (q = 0; q < L; ++q)
        residue[q] /= (double)trials;
    free(xm);
    free(cm);
    free(rm);
    return nmax;
}

/* ------------------------------------- Sec. 2.2, white noise (Reading 11b) */

/* One Philox4x32-10 block (Salmon et al., SC 2011): ten rounds of two 32 x 32 -> 64-bit
 * products of counter words with the round multipliers, whose high halves are mixed with
 * the other counter words and the round key, and a Weyl-sequence bump of the key between
 * rounds. */
void oracle_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* key increments */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    int r;
    for (r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* w (trials x L): realizations first .. first + trials - 1 for the seed, Reading 11b. */
void oracle_white_noise(uint64_t seed, int first, int trials, int64_t L, double *w)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double scale = 1.7320508075688772 / 8388608.0; /* sqrt(3) / 2^23 */
    int m;
    int64_t p;
    for (m = 0; m < trials; ++m) {
        for (p = 0; p < L; ++p) {
            const uint32_t ctr[4] = {(uint32_t)(p >> 2), (uint32_t)(first + m), 0u, 0u};
            uint32_t out[4];
            int32_t i;
            oracle_philox4x32_10(ctr, key, out);
            i = (int32_t)(2u * (out[p & 3] >> 9)) - 8388607;
            w[(int64_t)m * L + p] = (double)i * scale;
        }
    }
}

/* ---------------------------------------------------- Sec. 2.2, CEEMDAN */

/*
 * CEEMDAN of x (length L) with the noise realizations w (trials x L), Reading 12.
 * modes is K x L (slots past the produced count are zero), residue is L. The EMD
 * runs inside (noise modes, first modes) use the given stop rule and boundary.
 * Returns the number of modes produced.
 */
int oracle_ceemdan(const double *x, int64_t L, const double *w, int trials, double rel, int K,
                   int stop, int fixed_sifts, double sd_threshold, int max_sifts, int boundary,
                   int mirror_knots, double *modes, double *residue, int store_f32)
{
    const int KE = K - 1; /* noise modes E_1 .. E_{K-1} */
    size_t ne = (size_t)trials * (size_t)(KE > 0 ? KE : 1) * (size_t)L;
    double *E = (double *)malloc(ne * sizeof(double));
    double *wr = (double *)malloc((size_t)L * sizeof(double));
    double *r = (double *)malloc((size_t)L * sizeof(double));
    double *in = (double *)malloc((size_t)L * sizeof(double));
    double *c1 = (double *)malloc((size_t)L * sizeof(double));
    double *acc = (double *)malloc((size_t)L * sizeof(double));
    int32_t *sa = (int32_t *)malloc((size_t)L * sizeof(int32_t));
    int32_t *sb = (int32_t *)malloc((size_t)L * sizeof(int32_t));
    int k, m, n = 0;
    int64_t q;
    memset(modes, 0, (size_t)K * (size_t)L * sizeof(double));
    /* E_k(w^(m)) for k = 1 .. K-1: the EMD of each noise realization */
    if (KE > 0)
        for (m = 0; m < trials; ++m)
            oracle_emd(w + (int64_t)m * L, L, KE, stop, fixed_sifts, sd_threshold, max_sifts,
                       boundary, mirror_knots, E + (int64_t)m * KE * L, wr, NULL, store_f32);
    memcpy(r, x, (size_t)L * sizeof(double));
    for (k = 0; k < K; ++k) {
        double beta;
        if (!has_enough_extrema(r, L, sa, sb))
            break; /* r_k is the final residue */
        beta = rel * oracle_std(r, L);
        memset(acc, 0, (size_t)L * sizeof(double));
        for (m = 0; m < trials; ++m) {
            const double *e = k == 0 ? w + (int64_t)m * L : E + ((int64_t)m * KE + (k - 1)) * L;
            for (q = 0; q < L; ++q)
                in[q] = r[q] + beta * e[q];
            /* first mode of r_k + beta_k E_k(w^(m)); zero when it has no IMF */
            oracle_emd(in, L, 1, stop, fixed_sifts, sd_threshold, max_sifts, boundary,
                       mirror_knots, c1, wr, NULL, store_f32);
            for (q = 0; q < L; ++q)
                acc[q] += c1[q];
        }
        for (q = 0; q < L; ++q) {
            const double c = acc[q] / (double)trials;
            modes[(int64_t)k * L + q] = c;
            r[q] = r[q] - c; /* Step 3 */
        }
        ++n;
    }
    memcpy(residue, r, (size_t)L * sizeof(double));
    free(E);
    free(wr);
    free(r);
    free(in);
    free(c1);
    free(acc);
    free(sa);
    free(sb);
    return n;
}

/*
 * Serial-CEEMDAN (Sec. 3 with CEEMDAN as the decomposition F): serialize X,
 * CEEMDAN of x with w (trials x L), de-serialize. Returns the mode count.
 */
int oracle_serial_ceemdan(const double *X, int64_t M, int64_t N, int64_t D, int K, int stop,
                          int fixed_sifts, double sd_threshold, int max_sifts, int boundary,
                          int mirror_knots, int trials, double noise_rel_std, const double *w,
                          double *modes_out, double *residue_out, int store_f32)
{
    int64_t L = oracle_serial_length(M, N, D);
    double *x = (double *)malloc((size_t)L * sizeof(double));
    double *R = (double *)malloc((size_t)K * (size_t)L * sizeof(double));
    double *r = (double *)malloc((size_t)L * sizeof(double));
    int n;
    oracle_serialize(X, M, N, D, x);
    n = oracle_ceemdan(x, L, w, trials, noise_rel_std, K, stop, fixed_sifts, sd_threshold,
                       max_sifts, boundary, mirror_knots, R, r, store_f32);
    oracle_deserialize(R, K, M, N, D, modes_out);
    oracle_deserialize(r, 1, M, N, D, residue_out);
    free(x);
    free(R);
    free(r);
    return n;
}

/* ------------------------------------------------------ Sec. 3 end to end */

/*
 * Serial-EMD of one multi-signal (Sec. 3, the summary after Sec. 3.3):
 * serialize X (N signals of length M, D transition samples), decompose with
 * EMD (trials <= 1) or EEMD, de-serialize the IMFs and the residue.
 * imfs_out is K x N x M, residue_out is N x M. Returns the IMF count.
 */
int oracle_serial_emd(const double *X, int64_t M, int64_t N, int64_t D, int K, int stop,
                      int fixed_sifts, double sd_threshold, int max_sifts, int boundary,
                      int mirror_knots, int trials, double noise_rel_std, const double *w,
                      double *imfs_out, double *residue_out, int *sifts_per_imf, int store_f32)
{
    int64_t L = oracle_serial_length(M, N, D);
    double *x = (double *)malloc((size_t)L * sizeof(double));
    double *R = (double *)malloc((size_t)K * (size_t)L * sizeof(double));
    double *r = (double *)malloc((size_t)L * sizeof(double));
    int n;
    oracle_serialize(X, M, N, D, x);
    if (trials <= 1) {
        n = oracle_emd(x, L, K, stop, fixed_sifts, sd_threshold, max_sifts, boundary,
                       mirror_knots, R, r, sifts_per_imf, store_f32);
    } else {
        double beta = noise_rel_std * oracle_std(x, L);
        n = oracle_eemd(x, L, w, trials, beta, K, stop, fixed_sifts, sd_threshold,
                        max_sifts, boundary, mirror_knots, R, r, store_f32);
    }
    oracle_deserialize(R, K, M, N, D, imfs_out);
    oracle_deserialize(r, 1, M, N, D, residue_out);
    free(x);
    free(R);
    free(r);
    return n;
}
