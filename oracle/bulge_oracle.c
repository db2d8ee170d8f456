/*
 * ORACLE -- test infrastructure only.  Plain, slow, sequential FP64 reference
 * for the reduction of an upper-banded matrix to upper bidiagonal form by
 * Householder bulge chasing (Ringoot, Alomairy, Edelman, "Accelerating
 * Bidiagonalization of Banded Matrices through Memory-Aware Bulge-Chasing on
 * GPUs", arXiv 2510.12705).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the product library never
 * does, and it shares no code with it.
 *
 * What it computes (Section III, Algorithm 1; one row-bulge = Algorithm 2):
 *   for each bandwidth-reduction stage bw -> bw' = bw - d, d = min(TW, bw-1)
 *     for each sweep R = 0 .. n-2 (one sweep per row, in order)
 *       for each row-bulge s = 0, 1, ... of the sweep
 *         c  = R + bw' + s*bw   first column of the block; consecutive
 *                               row-bulges of a sweep are bw columns apart
 *                               (bw = bandwidth before the stage, Section III-A)
 *         m  = min(d+1, n-c)    reflector length; nothing to do if m <= 1
 *         r0 = R for s == 0, else c - bw: the row whose excess is removed
 *              (the first row-bulge of a sweep works on the sweep's own row)
 *         right reflector H from row r0, columns c..c+m-1; A <- A H on rows
 *             r0+1 .. c+m-1
 *         left reflector G from column c, rows c..c+m-1; A <- G A on columns
 *             c+1 .. min(n-1, c+m-1+bw)
 *   d = diag(A), e = superdiag(A).
 * Only the leading column / row of each bulge is annihilated; the remaining
 * fill is removed by the following sweeps (deferred bulges, Section III).
 *
 * Reflector generation (the paper defers its details to prior tile-QR work):
 * LAPACK xLARFG semantics, restated from its documented definition: with
 * alpha = x0 and xi = ||x(1:)||_2 (scaled norm), tau = 0 when xi == 0;
 * otherwise beta = -sign(alpha) hypot(alpha, xi) (sign(+-0) = +1),
 * tau = (beta - alpha)/beta, v = (1, x(1:)/(alpha - beta)), with the
 * documented rescaling loop when |beta| < safmin.
 *
 * The "order" argument selects the schedule: 0 = sequential (sweep-major),
 * L >= 1 = the paper's cycle schedule, in which sweep R executes its s-th
 * row-bulge in cycle L*R + s (Section III-A uses L = 3), processed within a
 * cycle from the highest sweep to the lowest; order = -L uses lag L on the
 * stages whose post-stage bandwidth is at least 2 and lag 3 on a stage that
 * ends at bandwidth 1 (the separation condition of Section III-A).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * result is the same on every host).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double flops;            /* reflector generation + application flops   */
    double elements;         /* elements touched: |right panel U left panel| per step */
    long long steps;         /* bulge steps with m >= 2                     */
    long long stages;        /* bandwidth-reduction stages executed         */
    long long fill_violations;  /* nonzeros found where the algorithm assumes zeros */
    long long out_of_band;      /* accesses outside the band-with-fill storage (must be 0) */
} oracle_counts;

/* Band-with-fill storage: element (i, j) at w[(i - j + up) + j * ld],
 * ld = up + lo + 1 with up = b + tw (upper fill), lo = tw (lower fill). */
typedef struct {
    double *w;
    int n, up, lo, ld;
    oracle_counts *cnt;
    double dummy;
} band_t;

static double *at(band_t *A, int i, int j)
{
    int off = i - j;
    if (i < 0 || j < 0 || i >= A->n || j >= A->n || off < -A->up || off > A->lo) {
        A->cnt->out_of_band++;
        A->dummy = 0.0;
        return &A->dummy;
    }
    return &A->w[(size_t)(off + A->up) + (size_t)j * (size_t)A->ld];
}

static int in_store(const band_t *A, int i, int j)
{
    int off = i - j;
    return i >= 0 && j >= 0 && i < A->n && j < A->n && off >= -A->up && off <= A->lo;
}

/* 2-norm with scaling by the largest magnitude (no overflow / underflow). */
static double scaled_norm(int m, const double *x)
{
    double scale = 0.0, ssq = 0.0;
    for (int k = 0; k < m; k++) {
        double a = fabs(x[k]);
        if (a > scale) scale = a;
    }
    if (scale == 0.0) return 0.0;
    for (int k = 0; k < m; k++) {
        double t = x[k] / scale;
        ssq += t * t;
    }
    return scale * sqrt(ssq);
}

/* xLARFG semantics.  x[0] = alpha on entry, x[0] = beta on exit; x[1..m-1]
 * becomes v[1..m-1] (v[0] = 1 implicit).  Returns tau. */
static double oracle_larfg(int m, double *x, double *flops)
{
    if (m <= 1) return 0.0;
    double alpha = x[0];
    double xnorm = scaled_norm(m - 1, x + 1);
    *flops += 3.0 * (m - 1);
    if (xnorm == 0.0) return 0.0;
    double beta = hypot(alpha, xnorm);
    if (alpha >= 0.0) beta = -beta;          /* beta = -sign(alpha)*hypot, sign(+-0)=+1 */
    const double safmin = DBL_MIN / DBL_EPSILON;
    int knt = 0;
    if (fabs(beta) < safmin) {
        const double rsafmn = 1.0 / safmin;
        do {
            knt++;
            for (int k = 1; k < m; k++) x[k] *= rsafmn;
            beta *= rsafmn;
            alpha *= rsafmn;
        } while (fabs(beta) < safmin && knt < 20);
        xnorm = scaled_norm(m - 1, x + 1);
        beta = hypot(alpha, xnorm);
        if (alpha >= 0.0) beta = -beta;
    }
    double tau = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int k = 1; k < m; k++) x[k] *= scal;
    *flops += (double)(m - 1) + 10.0;
    for (int j = 0; j < knt; j++) beta *= safmin;
    x[0] = beta;
    return tau;
}

/* One row-bulge of sweep R in the current stage (Algorithm 2). */
static void bulge_step(band_t *A, int bw, int d, int R, int s, double *v, int check)
{
    const int n = A->n;
    const int c = R + (bw - d) + s * bw;
    const int m = (d + 1 < n - c) ? d + 1 : n - c;
    if (m <= 1) return;
    const int r0 = (s == 0) ? R : c - bw;
    oracle_counts *cnt = A->cnt;
    cnt->steps++;

    /* rows above r0 must be zero in the block columns (deferred-bulge claim) */
    for (int i = r0 - 1; check && i >= 0 && in_store(A, i, c); i--)
        for (int k = 0; k < m; k++)
            if (in_store(A, i, c + k) && *at(A, i, c + k) != 0.0) cnt->fill_violations++;

    /* ---- right reflector: annihilate row r0, columns c+1 .. c+m-1 ---- */
    for (int k = 0; k < m; k++) v[k] = *at(A, r0, c + k);
    double tau = oracle_larfg(m, v, &cnt->flops);
    *at(A, r0, c) = v[0];
    for (int k = 1; k < m; k++) *at(A, r0, c + k) = 0.0;
    v[0] = 1.0;
    for (int r = r0 + 1; r <= c + m - 1; r++) {
        double w = 0.0;
        for (int k = 0; k < m; k++) w += *at(A, r, c + k) * v[k];
        w *= tau;
        for (int k = 0; k < m; k++) *at(A, r, c + k) -= w * v[k];
        cnt->flops += 4.0 * m;
    }

    /* ---- left reflector: annihilate column c, rows c+1 .. c+m-1 ---- */
    const int jmax = (c + m - 1 + bw < n - 1) ? c + m - 1 + bw : n - 1;
    /* columns right of jmax must be zero in the block rows */
    for (int j = jmax + 1; check && j < n && in_store(A, c, j); j++)
        for (int k = 0; k < m; k++)
            if (in_store(A, c + k, j) && *at(A, c + k, j) != 0.0) cnt->fill_violations++;
    for (int k = 0; k < m; k++) v[k] = *at(A, c + k, c);
    tau = oracle_larfg(m, v, &cnt->flops);
    *at(A, c, c) = v[0];
    for (int k = 1; k < m; k++) *at(A, c + k, c) = 0.0;
    v[0] = 1.0;
    for (int j = c + 1; j <= jmax; j++) {
        double w = 0.0;
        for (int k = 0; k < m; k++) w += v[k] * *at(A, c + k, j);
        w *= tau;
        for (int k = 0; k < m; k++) *at(A, c + k, j) -= w * v[k];
        cnt->flops += 4.0 * m;
    }

    /* |right panel U left panel|: right = rows r0..c+m-1 x m columns,
     * left = m rows x columns c..jmax, overlap = m x m */
    double right = (double)(c + m - r0) * m;
    double left = (double)m * (jmax - c + 1);
    cnt->elements += right + left - (double)m * m;
}

/* number of row-bulges of sweep R in a stage (bw, d) */
static int sweep_steps(int n, int bw, int d, int R)
{
    int c0 = R + (bw - d);
    if (c0 >= n - 1) return 0;
    return (n - 2 - c0) / bw + 1;
}

/*
 * Reduce the band.  ab: LAPACK 'U' band storage, A[i][j] = ab[(b+i-j) + j*ldab].
 * tw: inner tilewidth TW (>= 1).  order: 0 sequential, L >= 1 cycle schedule.
 * max_stages < 0: all stages.  max_steps < 0: no limit (a limit gives a
 * bounded timing sample; the output is then incomplete).
 * work_out (optional): receives the band-with-fill buffer, ld = b + 2*tw + 1,
 * element (i, j) at work_out[(i - j + b + tw) + j*ld] (b after clamping to n-1).
 * check_fill != 0: count nonzeros where the algorithm assumes zeros (slow).
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_band_to_bidiag(int n, int b, int tw, const double *ab, int ldab,
                          double *d_out, double *e_out, oracle_counts *cnt,
                          int order, int max_stages, long long max_steps,
                          double *work_out, int check_fill)
{
    if (n < 1 || b < 0 || tw < 1 || ldab < b + 1 || !ab || !d_out || !cnt) return -1;
    memset(cnt, 0, sizeof(*cnt));
    const int b_in = b;                 /* the caller's storage uses this b */
    if (b > n - 1) b = n - 1;
    band_t A;
    A.n = n;
    A.up = b + tw;
    A.lo = tw;
    A.ld = A.up + A.lo + 1;
    A.cnt = cnt;
    A.w = (double *)calloc((size_t)A.ld * (size_t)n, sizeof(double));
    double *v = (double *)malloc(sizeof(double) * (size_t)(tw + 2));
    int *nst = (int *)malloc(sizeof(int) * (size_t)(n > 1 ? n : 1));
    if (!A.w || !v || !nst) { free(A.w); free(v); free(nst); return -2; }
    /* b may have been clamped to n-1: read offsets 0..b with the caller's b */
    for (int j = 0; j < n; j++)
        for (int i = (j - b > 0 ? j - b : 0); i <= j; i++)
            *at(&A, i, j) = ab[(size_t)(b_in + i - j) + (size_t)j * (size_t)ldab];

    long long budget = max_steps;
    int bw = b, stage = 0;
    while (bw > 1 && (max_stages < 0 || stage < max_stages) && budget != 0) {
        const int d = (tw < bw - 1) ? tw : bw - 1;
        if (order == 0) {
            for (int R = 0; R < n - 1 && budget != 0; R++) {
                int ns = sweep_steps(n, bw, d, R);
                for (int s = 0; s < ns && budget != 0; s++) {
                    bulge_step(&A, bw, d, R, s, v, check_fill);
                    if (budget > 0) budget--;
                }
            }
        } else {
            /* Algorithm 1 cycle schedule: sweep R runs its s-th row-bulge in
             * cycle L*R + s; within a cycle, highest sweep first. */
            /* order < 0: lag |order| where the post-stage bandwidth is >= 2,
             * lag 3 on a stage that ends at bandwidth 1 (Section III-A) */
            const long long L = order > 0 ? order : ((bw - d >= 2) ? -order : 3);
            long long last = 0;
            for (int R = 0; R < n - 1; R++) {
                nst[R] = sweep_steps(n, bw, d, R);
                if (nst[R] > 0 && L * R + nst[R] > last) last = L * R + nst[R];
            }
            for (long long t = 0; t < last && budget != 0; t++) {
                long long rhi = t / L;
                if (rhi > n - 2) rhi = n - 2;
                for (long long R = rhi; R >= 0 && budget != 0; R--) {
                    long long s = t - L * R;
                    if (s >= nst[R]) break;   /* lower sweeps are further along */
                    bulge_step(&A, bw, d, (int)R, (int)s, v, check_fill);
                    if (budget > 0) budget--;
                }
            }
        }
        bw -= d;
        stage++;
    }
    cnt->stages = stage;
    for (int i = 0; i < n; i++) d_out[i] = *at(&A, i, i);
    if (e_out)
        for (int i = 0; i + 1 < n; i++) e_out[i] = *at(&A, i, i + 1);
    if (work_out) memcpy(work_out, A.w, sizeof(double) * (size_t)A.ld * (size_t)n);
    free(A.w);
    free(v);
    free(nst);
    return 0;
}

#ifdef _OPENMP
#include <omp.h>
/*
 * The cycle schedule of Section III-A with the row-bulges of one cycle run in
 * parallel: the paper's "synchronize parallel for" per cycle, on the host's
 * cores (OpenMP threads, a barrier after every cycle).  Lag 2 on the stages
 * whose post-stage bandwidth is at least 2 and lag 3 on a stage that ends at
 * bandwidth 1: under these lags the row-bulges of a cycle touch disjoint
 * elements, so the result is bitwise that of oracle_band_to_bidiag (each
 * row-bulge is the same bulge_step; every conflicting pair keeps its order).
 * A CPU baseline on all cores, not a reference: the tests pin it to the
 * sequential oracle.  max_steps >= 0 stops after the cycle in which that many
 * row-bulges were done.  *threads_used receives the thread count.
 */
int oracle_band_to_bidiag_omp(int n, int b, int tw, const double *ab, int ldab,
                              double *d_out, double *e_out, oracle_counts *cnt,
                              long long max_steps, int *threads_used)
{
    if (n < 1 || b < 0 || tw < 1 || ldab < b + 1 || !ab || !d_out || !cnt) return -1;
    memset(cnt, 0, sizeof(*cnt));
    const int b_in = b;
    if (b > n - 1) b = n - 1;
    band_t A;
    A.n = n;
    A.up = b + tw;
    A.lo = tw;
    A.ld = A.up + A.lo + 1;
    A.cnt = cnt;
    A.w = (double *)calloc((size_t)A.ld * (size_t)n, sizeof(double));
    int *nst = (int *)malloc(sizeof(int) * (size_t)(n > 1 ? n : 1));
    const int nthr = omp_get_max_threads();
    oracle_counts *tc = (oracle_counts *)calloc((size_t)nthr, sizeof(oracle_counts));
    double *vs = (double *)malloc(sizeof(double) * (size_t)(tw + 2) * (size_t)nthr);
    if (!A.w || !nst || !tc || !vs) { free(A.w); free(nst); free(tc); free(vs); return -2; }
    for (int j = 0; j < n; j++)
        for (int i = (j - b > 0 ? j - b : 0); i <= j; i++)
            *at(&A, i, j) = ab[(size_t)(b_in + i - j) + (size_t)j * (size_t)ldab];

    long long done = 0;
    int bw = b, stage = 0;
    while (bw > 1 && (max_steps < 0 || done < max_steps)) {
        const int d = (tw < bw - 1) ? tw : bw - 1;
        const long long L = (bw - d >= 2) ? 2 : 3;
        long long last = 0;
        for (int R = 0; R < n - 1; R++) {
            nst[R] = sweep_steps(n, bw, d, R);
            if (nst[R] > 0 && L * R + nst[R] > last) last = L * R + nst[R];
        }
        long long base = done;
        #pragma omp parallel
        {
            const int me = omp_get_thread_num();
            band_t Am = A;                    /* own counters and out-of-band slot */
            Am.cnt = &tc[me];
            double *v = vs + (size_t)(tw + 2) * (size_t)me;
            long long mine = base;            /* the same count in every thread */
            for (long long t = 0; t < last; t++) {
                if (max_steps >= 0 && mine >= max_steps) break;
                long long rhi = t / L;
                if (rhi > n - 2) rhi = n - 2;
                long long rlo = rhi + 1;      /* the sweeps with a row-bulge in this cycle */
                while (rlo - 1 >= 0 && t - L * (rlo - 1) < nst[rlo - 1]) rlo--;
                #pragma omp for schedule(static)
                for (long long R = rlo; R <= rhi; R++)
                    bulge_step(&Am, bw, d, (int)R, (int)(t - L * R), v, 0);
                mine += rhi - rlo + 1;
            }
            if (me == 0) done = mine;
        }
        bw -= d;
        stage++;
    }
    for (int k = 0; k < nthr; k++) {
        cnt->flops += tc[k].flops;
        cnt->elements += tc[k].elements;
        cnt->steps += tc[k].steps;
        cnt->out_of_band += tc[k].out_of_band;
    }
    cnt->stages = stage;
    for (int i = 0; i < n; i++) d_out[i] = *at(&A, i, i);
    if (e_out)
        for (int i = 0; i + 1 < n; i++) e_out[i] = *at(&A, i, i + 1);
    if (threads_used) *threads_used = nthr;
    free(A.w);
    free(nst);
    free(tc);
    free(vs);
    return 0;
}
#endif

/*
 * Singular values of the upper bidiagonal B(d, e) by Sturm-count bisection
 * on its Golub-Kahan form: the 2n x 2n symmetric tridiagonal matrix with zero
 * diagonal and off-diagonal (d0, e0, d1, e1, ..., d_{n-1}), whose eigenvalues
 * are +-sigma_k.  sigma_out receives the n values in descending order.
 */
static long long gk_count_below(int n, const double *d, const double *e, double x,
                                double pivmin)
{
    /* number of eigenvalues of the Golub-Kahan matrix smaller than x */
    long long neg = 0;
    double q = -x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) neg++;
    for (int k = 1; k < 2 * n; k++) {
        double off = (k & 1) ? d[(k - 1) / 2] : e[(k - 2) / 2];
        q = -x - off * off / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) neg++;
    }
    return neg;
}

/* #{sigma < x} of the bidiagonal (d, e) for x > 0: the negative pivots of the
 * Golub-Kahan matrix shifted by x, minus n (exported for the tests) */
long long oracle_gk_count(int n, const double *d, const double *e, double x, double pivmin)
{
    return gk_count_below(n, d, e, x, pivmin) - n;
}

int oracle_bidiag_sigma(int n, const double *d, const double *e, double *sigma_out)
{
    if (n < 1) return -1;
    double bound = 0.0, maxoff = 0.0;
    for (int i = 0; i < n; i++) {
        double r = fabs(d[i]) + (i + 1 < n ? fabs(e[i]) : 0.0);
        double l = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
        if (r > bound) bound = r;
        if (l > bound) bound = l;
        if (fabs(d[i]) > maxoff) maxoff = fabs(d[i]);
        if (i + 1 < n && fabs(e[i]) > maxoff) maxoff = fabs(e[i]);
    }
    if (bound == 0.0) {
        for (int i = 0; i < n; i++) sigma_out[i] = 0.0;
        return 0;
    }
    const double pivmin = DBL_MIN * (maxoff * maxoff > 1.0 ? maxoff * maxoff : 1.0);
    /* sigma_k (k-th largest): the smallest x with #{sigma < x} >= n - k */
    for (int k = 0; k < n; k++) {
        long long target = n - k;          /* need count_below(x) - n >= target */
        double lo = 0.0, hi = bound * (1.0 + 4.0 * DBL_EPSILON) + DBL_MIN;
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            long long cntb = gk_count_below(n, d, e, mid, pivmin) - n;
            if (cntb >= target) hi = mid; else lo = mid;
            if (hi - lo <= 2.0 * DBL_EPSILON * hi) break;
        }
        sigma_out[k] = 0.5 * (lo + hi);
    }
    return 0;
}

/*
 * One-sided Jacobi SVD (Hestenes) of a dense n x n column-major matrix,
 * brute force for small n.  sigma_out: descending.  a is overwritten.
 */
int oracle_jacobi_sigma(int n, double *a, double *sigma_out)
{
    if (n < 1) return -1;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double *ap = a + (size_t)p * n, *aq = a + (size_t)q * n;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < n; i++) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (gamma == 0.0) continue;
                double rel = fabs(gamma) / sqrt(alpha * beta);
                if (rel > off) off = rel;
                if (rel < 1e-15) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < n; i++) {
                    double x = ap[i], y = aq[i];
                    ap[i] = cs * x - sn * y;
                    aq[i] = sn * x + cs * y;
                }
            }
        }
        if (off < 1e-15) break;
    }
    for (int p = 0; p < n; p++) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += a[(size_t)p * n + i] * a[(size_t)p * n + i];
        sigma_out[p] = sqrt(s);
    }
    /* sort descending (insertion sort, n is small) */
    for (int i = 1; i < n; i++) {
        double x = sigma_out[i];
        int j = i - 1;
        while (j >= 0 && sigma_out[j] < x) { sigma_out[j + 1] = sigma_out[j]; j--; }
        sigma_out[j + 1] = x;
    }
    return 0;
}
