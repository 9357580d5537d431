/*
 * FP64 CPU oracle for the 2D complex-to-complex discrete Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the test suite, the smoke check and the CPU-baseline leg of the bench
 * may load.  The library product (the CUDA path) never calls it, includes it
 * or shares any code, table or constant with it.
 *
 * What it computes.  The unnormalised DFT,
 *     X[k] = sum_{j<n} x[j] * exp(dir * 2*pi*i * j*k / n),   dir = -1 forward,
 * and its 2D form, a 1D DFT along every row (contiguous axis, length nx)
 * followed by a 1D DFT along every column (length ny) -- the row-then-column
 * decomposition of the paper's Section 5 (Fig. 6).  The paper prints neither
 * a sign convention nor a normalisation; this oracle uses the forward sign -1
 * and no scaling in either direction.
 *
 * How.  oracle_fft1d_batch and oracle_fft2d use the plain recursive radix-2
 * Cooley-Tukey split of Section 2.2 (the divide-and-conquer form the paper
 * describes before its iterative Listing 1): X[k] = E[k] + w^k O[k] and
 * X[k+n/2] = E[k] - w^k O[k] with w = exp(dir*2*pi*i/n), every twiddle
 * evaluated directly from the integer ratio k/n in double precision, never by
 * repeated multiplication.  oracle_dft1d_brute / oracle_dft2d_brute are the
 * O(N^2) definition with the phase index (j*k mod n) reduced in integers; the
 * sampled-output functions combine the definition along one axis with the
 * recursive transform along the other, for spot checks of transforms too large
 * to recompute whole; oracle_dft1d_bins evaluates single bins of a long 1D
 * transform from the definition.  oracle_fft1d_any / oracle_fft2d_any
 * take any length: the same recursion split by the smallest prime factor
 * instead of 2, with prime lengths from the definition.
 *
 * Data.  Interleaved complex128 (re, im) arrays, row-major [batch][ny][nx].
 * Inputs are never modified.  Every function returns 0 on success and a
 * negative value on a bad argument (n not a power of two, NULL pointer).
 *
 * Mutants.  Building with -DORACLE_MUTANT=<k> plants one deliberate mistake
 * (see the MUTANT markers); the test suite uses those builds to show that the
 * pins around this oracle catch each kind of mistake.  The default build
 * (ORACLE_MUTANT undefined or 0) has none.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double re, im;
} cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

/* exp(dir * 2*pi*i * k / n) straight from the ratio k/n. */
static cplx root(long k, long n, int dir) {
#if ORACLE_MUTANT == 3
    k = k + 1; /* MUTANT 3: off-by-one twiddle exponent */
#endif
    double a = TWO_PI * (double)k / (double)n;
    cplx w;
    w.re = cos(a);
#if ORACLE_MUTANT == 1
    w.im = -(double)dir * sin(a); /* MUTANT 1: twiddle sign flipped */
#else
    w.im = (double)dir * sin(a);
#endif
    return w;
}

static cplx cmul(cplx a, cplx b) {
    cplx c;
    c.re = a.re * b.re - a.im * b.im;
    c.im = a.re * b.im + a.im * b.re;
    return c;
}

/*
 * Recursive radix-2 decimation in time: the n inputs x[0], x[s], x[2s], ...
 * are transformed into X[0..n).  Even-indexed inputs go to X[0..n/2), odd ones
 * to X[n/2..n), then the butterflies of Section 2.2 combine the two halves.
 */
static void ct_rec(const cplx *x, long s, cplx *X, long n, int dir) {
    if (n == 1) {
        X[0] = x[0];
        return;
    }
    long h = n / 2;
    ct_rec(x, 2 * s, X, h, dir);
    ct_rec(x + s, 2 * s, X + h, h, dir);
    for (long k = 0; k < h; ++k) {
        cplx e = X[k];
        cplx o = cmul(root(k, n, dir), X[k + h]);
#if ORACLE_MUTANT == 2
        o.re = 0.0 * o.re; /* MUTANT 2: the odd half's real part dropped */
#endif
        X[k].re = e.re + o.re;
        X[k].im = e.im + o.im;
        X[k + h].re = e.re - o.re;
        X[k + h].im = e.im - o.im;
    }
}

/* One length-n transform of a contiguous vector (out may not alias in). */
static void fft1d(const cplx *in, cplx *out, long n, int dir) {
    ct_rec(in, 1, out, n, dir);
}

/*
 * howmany independent length-n transforms of contiguous vectors, the rows of
 * a [howmany][n] array.  threads > 1 spreads rows over OpenMP threads; each
 * row is computed exactly as in the serial case.
 */
int oracle_fft1d_batch(const double *in, double *out, long n, long howmany, int dir,
                       int threads) {
    if (!in || !out || !is_pow2(n) || howmany < 0 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (long r = 0; r < howmany; ++r) {
        fft1d(x + r * n, X + r * n, n, dir);
    }
    return 0;
}

/*
 * 2D transform of each [ny][nx] slice of a [batch][ny][nx] array: the 1D DFT
 * along every row, then along every column (Section 5, Fig. 6).  Output is in
 * natural [ky][kx] order, never left transposed.
 */
int oracle_fft2d(const double *in, double *out, long nx, long ny, long batch, int dir,
                 int threads) {
    if (!in || !out || !is_pow2(nx) || !is_pow2(ny) || batch < 0 || (dir != 1 && dir != -1))
        return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
    long N = nx * ny;
#if ORACLE_MUTANT == 6
    /* MUTANT 6: conjugated input */
    cplx *xc = (cplx *)malloc(sizeof(cplx) * (size_t)(N * batch));
    for (long i = 0; i < N * batch; ++i) {
        xc[i].re = x[i].re;
        xc[i].im = -x[i].im;
    }
    x = xc;
#endif
    /* rows */
#pragma omp parallel for num_threads(threads) schedule(static)
    for (long r = 0; r < ny * batch; ++r) {
        fft1d(x + r * nx, X + r * nx, nx, dir);
    }
#if ORACLE_MUTANT == 5
    return 0; /* MUTANT 5: column pass dropped */
#endif
    /* columns: gather, transform, scatter */
#pragma omp parallel num_threads(threads)
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
        cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
#pragma omp for schedule(static)
        for (long c = 0; c < nx * batch; ++c) {
            long b = c / nx, xi = c % nx;
            cplx *base = X + b * N;
#if ORACLE_MUTANT == 4
            long len = nx; /* MUTANT 4: row length used as the column length */
            if (len > ny) len = ny;
#else
            long len = ny;
#endif
            for (long y = 0; y < len; ++y) col[y] = base[y * nx + xi];
            fft1d(col, res, len, dir);
            for (long y = 0; y < len; ++y) base[y * nx + xi] = res[y];
        }
        free(col);
        free(res);
    }
#if ORACLE_MUTANT == 6
    free(xc);
#endif
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Any length n >= 1 (not only powers of two).                               */
/* ------------------------------------------------------------------------ */

static long smallest_prime_factor(long n) {
    if (n % 2 == 0) return 2;
    for (long p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

static cplx root_exact(long long p, long long n, int dir);

/*
 * Recursive mixed-radix Cooley-Tukey, decimation in time by the smallest
 * prime factor p of n (the radix-2 split of Section 2.2 with 2 replaced by
 * p): with m = n/p and Y_r the length-m transform of x[r], x[r+p], ...,
 *     X[k] = sum_{r<p} exp(dir*2*pi*i*r*k/n) * Y_r[k mod m].
 * A prime length is evaluated from the definition.  Inputs x[0], x[s], ...
 */
static void ct_any(const cplx *x, long s, cplx *X, long n, int dir) {
    const long p = smallest_prime_factor(n);
    if (p == n) {
        for (long k = 0; k < n; ++k) {
            double sr = 0.0, si = 0.0;
            for (long j = 0; j < n; ++j) {
                cplx w = root_exact(((long long)j * k) % n, n, dir);
                cplx v = x[j * s];
                sr += v.re * w.re - v.im * w.im;
                si += v.re * w.im + v.im * w.re;
            }
            X[k].re = sr;
            X[k].im = si;
        }
        return;
    }
    const long m = n / p;
    cplx *Y = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (long r = 0; r < p; ++r) ct_any(x + r * s, s * p, Y + r * m, m, dir);
    for (long k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (long r = 0; r < p; ++r) {
#if ORACLE_MUTANT == 9
            cplx w = root_exact(((long long)r * k) % m, n, dir); /* MUTANT 9: phase reduced mod m */
#else
            cplx w = root_exact(((long long)r * k) % n, n, dir);
#endif
            cplx v = Y[r * m + k % m];
            sr += v.re * w.re - v.im * w.im;
            si += v.re * w.im + v.im * w.re;
        }
        X[k].re = sr;
        X[k].im = si;
    }
    free(Y);
}

/* howmany transforms of any length n >= 1 along contiguous rows. */
int oracle_fft1d_any(const double *in, double *out, long n, long howmany, int dir, int threads) {
    if (!in || !out || n < 1 || howmany < 0 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (long r = 0; r < howmany; ++r) ct_any(x + r * n, 1, X + r * n, n, dir);
    return 0;
}

/* 2D transform of each [ny][nx] slice, any nx, ny >= 1: rows, then columns. */
int oracle_fft2d_any(const double *in, double *out, long nx, long ny, long batch, int dir, int threads) {
    if (!in || !out || nx < 1 || ny < 1 || batch < 0 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
    const long N = nx * ny;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (long r = 0; r < ny * batch; ++r) ct_any(x + r * nx, 1, X + r * nx, nx, dir);
#pragma omp parallel num_threads(threads)
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
        cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
#pragma omp for schedule(static)
        for (long c = 0; c < nx * batch; ++c) {
            const long b = c / nx, xi = c % nx;
            cplx *base = X + b * N;
            for (long y = 0; y < ny; ++y) col[y] = base[y * nx + xi];
            ct_any(col, 1, res, ny, dir);
            for (long y = 0; y < ny; ++y) base[y * nx + xi] = res[y];
        }
        free(col);
        free(res);
    }
    return 0;
}

/* exp(dir*2*pi*i*p/n) for an already reduced integer phase index 0 <= p < n. */
static cplx root_exact(long long p, long long n, int dir) {
    double a = TWO_PI * (double)p / (double)n;
    cplx w;
    w.re = cos(a);
#if ORACLE_MUTANT == 7
    w.im = -(double)dir * sin(a); /* MUTANT 7: brute-force sign flipped */
#else
    w.im = (double)dir * sin(a);
#endif
    return w;
}

/* The O(n^2) definition of the 1D DFT, phase index (j*k) mod n in integers. */
int oracle_dft1d_brute(const double *in, double *out, long n, int dir) {
    if (!in || !out || n < 1 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    for (long k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (long j = 0; j < n; ++j) {
            cplx w = root_exact(((long long)j * k) % n, n, dir);
            sr += x[j].re * w.re - x[j].im * w.im;
            si += x[j].re * w.im + x[j].im * w.re;
        }
        X[k].re = sr;
        X[k].im = si;
    }
    return 0;
}

/*
 * The O(N^2) definition of the 2D DFT of one [ny][nx] array:
 *   X[ky][kx] = sum_y sum_x x[y][x] exp(dir*2*pi*i*((ky*y mod ny)/ny + (kx*x mod nx)/nx)).
 */
int oracle_dft2d_brute(const double *in, double *out, long nx, long ny, int dir) {
    if (!in || !out || nx < 1 || ny < 1 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    for (long ky = 0; ky < ny; ++ky) {
        for (long kx = 0; kx < nx; ++kx) {
            double sr = 0.0, si = 0.0;
            for (long y = 0; y < ny; ++y) {
                for (long xi = 0; xi < nx; ++xi) {
                    long long py = ((long long)ky * y) % ny;
                    long long px = ((long long)kx * xi) % nx;
                    /* common denominator nx*ny keeps the phase an exact integer ratio */
                    long long p = (py * nx + px * ny) % ((long long)nx * ny);
                    cplx w = root_exact(p, (long long)nx * ny, dir);
                    cplx v = x[y * nx + xi];
                    sr += v.re * w.re - v.im * w.im;
                    si += v.re * w.im + v.im * w.re;
                }
            }
            X[ky * nx + kx].re = sr;
            X[ky * nx + kx].im = si;
        }
    }
    return 0;
}

/*
 * Selected output rows of the 2D transform of one [ny][nx] array:
 *   X[ky][:] = FFT_x( sum_y x[y][:] * exp(dir*2*pi*i*(ky*y mod ny)/ny) )
 * -- the definition along y (one pass over the data per requested row), then
 * the recursive transform along x.  out is [nk][nx].
 */
int oracle_fft2d_rows(const double *in, double *out, long nx, long ny, const long *ky,
                      long nk, int dir, int threads) {
    if (!in || !out || !ky || !is_pow2(nx) || ny < 1 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
    for (long t = 0; t < nk; ++t)
        if (ky[t] < 0 || ky[t] >= ny) return -1;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (long t = 0; t < nk; ++t) {
        cplx *acc = (cplx *)calloc((size_t)nx, sizeof(cplx));
        for (long y = 0; y < ny; ++y) {
            cplx w = root_exact(((long long)ky[t] * y) % ny, ny, dir);
            const cplx *row = x + y * nx;
            for (long xi = 0; xi < nx; ++xi) {
                acc[xi].re += row[xi].re * w.re - row[xi].im * w.im;
                acc[xi].im += row[xi].re * w.im + row[xi].im * w.re;
            }
        }
        fft1d(acc, X + t * nx, nx, dir);
        free(acc);
    }
    return 0;
}

/*
 * Selected output columns of the 2D transform of one [ny][nx] array:
 *   X[:][kx] = FFT_y( sum_x x[:][x] * exp(dir*2*pi*i*(kx*x mod nx)/nx) ).
 * out is [nk][ny] (column t stored contiguously).
 */
int oracle_fft2d_cols(const double *in, double *out, long nx, long ny, const long *kx,
                      long nk, int dir, int threads) {
    if (!in || !out || !kx || !is_pow2(ny) || nx < 1 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
    for (long t = 0; t < nk; ++t)
        if (kx[t] < 0 || kx[t] >= nx) return -1;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (long t = 0; t < nk; ++t) {
        cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)nx);
        cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
        for (long xi = 0; xi < nx; ++xi) w[xi] = root_exact(((long long)kx[t] * xi) % nx, nx, dir);
        for (long y = 0; y < ny; ++y) {
            double sr = 0.0, si = 0.0;
            const cplx *row = x + y * nx;
            for (long xi = 0; xi < nx; ++xi) {
                sr += row[xi].re * w[xi].re - row[xi].im * w[xi].im;
                si += row[xi].re * w[xi].im + row[xi].im * w[xi].re;
            }
            acc[y].re = sr;
            acc[y].im = si;
        }
        fft1d(acc, X + t * ny, ny, dir);
        free(w);
        free(acc);
    }
    return 0;
}

/*
 * Selected bins of one length-n 1D transform, straight from the definition:
 *   X[k] = sum_{j<n} x[j] * exp(dir*2*pi*i*(j*k mod n)/n),  k in bins[0..nb).
 * One O(n) pass per bin, for spot checks of 1D transforms too long to
 * recompute whole with the recursive form (n up to 2^26).  out is [nb].
 */
int oracle_dft1d_bins(const double *in, double *out, long n, const long *bins, long nb, int dir,
                      int threads) {
    if (!in || !out || !bins || n < 1 || nb < 0 || (dir != 1 && dir != -1)) return -1;
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    if (threads < 1) threads = 1;
    for (long t = 0; t < nb; ++t)
        if (bins[t] < 0 || bins[t] >= n) return -1;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (long t = 0; t < nb; ++t) {
        long long k = bins[t];
#if ORACLE_MUTANT == 8
        k = (k + 1) % n; /* MUTANT 8: the neighbouring bin */
#endif
        double sr = 0.0, si = 0.0;
        for (long j = 0; j < n; ++j) {
            cplx w = root_exact(((long long)j * k) % n, n, dir);
            sr += x[j].re * w.re - x[j].im * w.im;
            si += x[j].re * w.im + x[j].im * w.re;
        }
        X[t].re = sr;
        X[t].im = si;
    }
    return 0;
}

/* Number of OpenMP threads available (1 when built without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
