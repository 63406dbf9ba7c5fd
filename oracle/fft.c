/*
 * Oracle FFT: a plain recursive mixed-radix Cooley-Tukey transform
 * (decimation in time, any factor, smallest prime first) and a brute-force
 * direct DFT.  Sec. 2.4 discretizes the fields by truncated Fourier series
 * evaluated with the FFT; this file is that FFT written from its definition
 *
 *     X[k] = sum_{j=0}^{n-1} x[j] exp(sign * 2 pi i j k / n),
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* exp(sign*2*pi*i*j/n) for j = 0..n-1, evaluated in long double. */
static double complex *twiddle_table(long n, int sign)
{
    double complex *w = malloc(sizeof(double complex) * (size_t)n);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (long j = 0; j < n; ++j) {
        long double a = two_pi * (long double)j / (long double)n;
        w[j] = (double)cosl(a) + (double)(sign * sinl(a)) * I;
    }
    return w;
}

static long smallest_factor(long n)
{
    for (long p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * out[k] = sum_{j<n} in[j*stride] * W^{j k (N/n)},  W = tab[1] = exp(sign 2 pi i / N).
 * Split j = p*j' + r: the p sub-sequences are transformed recursively into
 * out[r*m .. r*m+m-1] and combined as
 *     X[k + q m] = sum_r W_n^{r k} W_p^{r q} Y_r[k].
 */
static void fft_rec(const double complex *in, long stride, double complex *out,
                    long n, long N, const double complex *tab)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    long p = smallest_factor(n);
    long m = n / p;
    for (long r = 0; r < p; ++r)
        fft_rec(in + r * stride, stride * p, out + r * m, m, N, tab);

    long step = N / n; /* W_n^x = tab[x * step mod N] */
    double complex small[16];
    double complex *t = p <= 8 ? small : malloc(sizeof(double complex) * (size_t)p * 2);
    double complex *o = t + p;
    for (long k = 0; k < m; ++k) {
        for (long r = 0; r < p; ++r)
            t[r] = out[r * m + k] * tab[(r * k * step) % N];
        for (long q = 0; q < p; ++q) {
            double complex acc = 0;
            for (long r = 0; r < p; ++r)
                acc += t[r] * tab[(r * q * m * step) % N];
            o[q] = acc;
        }
        for (long q = 0; q < p; ++q) out[k + q * m] = o[q];
    }
    if (t != small) free(t);
}

/* Transform `count` lines of length n; line l starts at data + l*ldist,
 * elements are `stride` apart. */
static void fft_lines(double complex *data, long n, long stride, long count,
                      long ldist, int sign)
{
    double complex *tab = twiddle_table(n, sign);
    /* the lines are independent: in the OpenMP build (timing only) each
     * thread takes a share of them with its own buffers */
#pragma omp parallel
    {
        double complex *a = malloc(sizeof(double complex) * (size_t)n * 2);
        double complex *b = a + n;
#pragma omp for schedule(static)
        for (long l = 0; l < count; ++l) {
            double complex *line = data + l * ldist;
            for (long j = 0; j < n; ++j) a[j] = line[j * stride];
            fft_rec(a, 1, b, n, n, tab);
            for (long j = 0; j < n; ++j) line[j * stride] = b[j];
        }
        free(a);
    }
    free(tab);
}

void orc_fft1(int n, double complex *data, int sign)
{
    fft_lines(data, n, 1, 1, n, sign);
}

/* Unnormalized forward transform of a real field: out = sum x e^{-i k.x}
 * over the half spectrum out[z][y][0..nx/2]. */
void orc_fft3_r2c(int nx, int ny, int nz, const double *in, double complex *out)
{
    long hx = nx / 2 + 1;
    double complex *tab = twiddle_table(nx, -1);
#pragma omp parallel
    {
        double complex *line = malloc(sizeof(double complex) * (size_t)nx);
        double complex *res = malloc(sizeof(double complex) * (size_t)nx);
#pragma omp for schedule(static)
        for (long zy = 0; zy < (long)nz * ny; ++zy) {
            for (long x = 0; x < nx; ++x) line[x] = in[zy * nx + x];
            fft_rec(line, 1, res, nx, nx, tab);
            for (long x = 0; x < hx; ++x) out[zy * hx + x] = res[x];
        }
        free(res);
        free(line);
    }
    free(tab);
    /* y lines: for each z plane, hx lines of stride hx */
    for (long z = 0; z < nz; ++z)
        fft_lines(out + z * ny * hx, ny, hx, hx, 1, -1);
    /* z lines: ny*hx lines of stride ny*hx */
    fft_lines(out, nz, (long)ny * hx, (long)ny * hx, 1, -1);
}

/* Unnormalized inverse: out(x) = sum over the full spectrum of X e^{+i k.x},
 * the missing half filled by Hermitian symmetry X(-k) = conj X(k). */
void orc_fft3_c2r(int nx, int ny, int nz, const double complex *in, double *out)
{
    long hx = nx / 2 + 1;
    long nh = (long)nz * ny * hx;
    double complex *w = malloc(sizeof(double complex) * (size_t)nh);
    memcpy(w, in, sizeof(double complex) * (size_t)nh);
    fft_lines(w, nz, (long)ny * hx, (long)ny * hx, 1, +1);
    for (long z = 0; z < nz; ++z)
        fft_lines(w + z * ny * hx, ny, hx, hx, 1, +1);
    double complex *tab = twiddle_table(nx, +1);
#pragma omp parallel
    {
        double complex *line = malloc(sizeof(double complex) * (size_t)nx);
        double complex *res = malloc(sizeof(double complex) * (size_t)nx);
#pragma omp for schedule(static)
        for (long zy = 0; zy < (long)nz * ny; ++zy) {
            const double complex *h = w + zy * hx;
            for (long x = 0; x < hx; ++x) line[x] = h[x];
            for (long x = hx; x < nx; ++x) line[x] = conj(h[nx - x]);
            fft_rec(line, 1, res, nx, nx, tab);
            for (long x = 0; x < nx; ++x) out[zy * nx + x] = creal(res[x]);
        }
        free(res);
        free(line);
    }
    free(tab);
    free(w);
}

/* Brute-force direct DFT of a real field onto the half spectrum (O(N^2)). */
void orc_dft3_r2c(int nx, int ny, int nz, const double *in, double complex *out)
{
    long hx = nx / 2 + 1;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (long kz = 0; kz < nz; ++kz)
        for (long ky = 0; ky < ny; ++ky)
            for (long kx = 0; kx < hx; ++kx) {
                long double re = 0, im = 0;
                for (long z = 0; z < nz; ++z)
                    for (long y = 0; y < ny; ++y)
                        for (long x = 0; x < nx; ++x) {
                            /* phase reduced exactly in integers first */
                            long double ph =
                                (long double)((kx * x) % nx) / nx +
                                (long double)((ky * y) % ny) / ny +
                                (long double)((kz * z) % nz) / nz;
                            long double a = -two_pi * ph;
                            long double v = in[(z * ny + y) * nx + x];
                            re += v * cosl(a);
                            im += v * sinl(a);
                        }
                out[(kz * ny + ky) * hx + kx] = (double)re + (double)im * I;
            }
}
