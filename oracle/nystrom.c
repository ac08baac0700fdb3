/*
 * Oracle: plain, slow, FP64 direct Nystrom sums for the homogeneous-medium
 * Fredholm operators of the radiative transfer equation (Fan, An, Ying,
 * "Fast algorithms for integral formulations of steady-state radiative
 * transfer equation").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a host library that
 * only the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark load.  It shares no code with the CUDA path: no headers, no
 * tables, no helpers.
 *
 * What it evaluates (no FFT, no blocking, no symmetry tricks):
 *
 *  2D (Sec. 3.1.1, Eq. ani_2d_operator and Sec. 3.3, Eq. ani_discretization):
 *    out[(i,k)] = sum_j sum_{k'=-Li..Li} Kt[(i,k),(j,k')] * phi[(j,k')],
 *    k = -Lo..Lo, with the matrix of the kernel
 *      Kt(x,k,y,k') = kappa(x-y) * exp(i (k'-k) theta(x-y)),
 *      kappa(r)     = exp(-mu_t |r|) / (2 pi |r|)      (Sec. 2.3.1, d = 2),
 *    theta(r) the polar angle of r.  Off the diagonal the entry is the kernel
 *    at the two cell centres times the cell area h^2; on the diagonal it is
 *    the integral of the kernel over the cell (Sec. 2.3, after
 *    Eq. iso_discretization), passed in as D[m] = int_cell kappa e^{i m theta},
 *    m = k' - k.  D is real (the cell is symmetric under reflections).
 *
 *  3D isotropic (Sec. 2.3.1, d = 3):
 *    out[i] = sum_j Kt[i,j] phi[j],  kappa(r) = exp(-mu_t |r|)/(4 pi |r|^2),
 *    off-diagonal h^3 kappa(x_i - x_j), diagonal D (cell integral).
 *
 *  Cell centres x_i = ((i1 + 1/2) h, (i2 + 1/2) h [, (i3 + 1/2) h]).
 *
 *  Complex arrays are interleaved (re, im) doubles.  2D mode-major layout:
 *  phi[((k + Li) * N + j) * 2 + {0,1}], N = n*n, j = j2 * n + j1 (x fastest).
 *  3D layout: phi[(j3 * n + j2) * n + j1].
 *
 *  `rows` (optional, may be NULL) restricts the output to the listed cells;
 *  out then holds nrows cells per mode in the order given.
 */
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* kappa for d = 2 at distance r > 0 */
static double kappa2(double mu_t, double r) { return exp(-mu_t * r) / (2.0 * M_PI * r); }

/* kappa for d = 3 at distance r > 0 */
static double kappa3(double mu_t, double r) { return exp(-mu_t * r) / (4.0 * M_PI * r * r); }

void oracle_Ktilde_2d(int n, double h, double mu_t, int Lo, int Li,
                      const double *D /* D[m + Lo + Li], m = -(Lo+Li)..(Lo+Li) */,
                      const double *phi, double *out, const int *rows, int nrows)
{
    const long N = (long)n * n;
    const int Mo = 2 * Lo + 1, Mi = 2 * Li + 1;
    const long nout = rows ? nrows : N;
    #pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < nout; ++r) {
        const long i = rows ? rows[r] : r;
        const int i1 = (int)(i % n), i2 = (int)(i / n);
        const double xi1 = (i1 + 0.5) * h, xi2 = (i2 + 0.5) * h;
        for (int ko = 0; ko < Mo; ++ko) {
            const int k = ko - Lo;
            double acc_re = 0.0, acc_im = 0.0;
            for (long j = 0; j < N; ++j) {
                const int j1 = (int)(j % n), j2 = (int)(j / n);
                for (int ki = 0; ki < Mi; ++ki) {
                    const int kp = ki - Li;
                    const double p_re = phi[((long)ki * N + j) * 2 + 0];
                    const double p_im = phi[((long)ki * N + j) * 2 + 1];
                    double e_re, e_im; /* matrix entry */
                    if (j == i) {
                        e_re = D[(kp - k) + Lo + Li];
                        e_im = 0.0;
                    } else {
                        const double d1 = xi1 - (j1 + 0.5) * h;
                        const double d2 = xi2 - (j2 + 0.5) * h;
                        const double rr = sqrt(d1 * d1 + d2 * d2);
                        const double th = atan2(d2, d1);
                        const double w = h * h * kappa2(mu_t, rr);
                        e_re = w * cos((kp - k) * th);
                        e_im = w * sin((kp - k) * th);
                    }
                    acc_re += e_re * p_re - e_im * p_im;
                    acc_im += e_re * p_im + e_im * p_re;
                }
            }
            out[((long)ko * nout + r) * 2 + 0] = acc_re;
            out[((long)ko * nout + r) * 2 + 1] = acc_im;
        }
    }
}

/* Dense matrix of the same operator, rows (i,k), columns (j,k'), mode-major:
 * A[((ko*N + i) * (Mi*N) + (ki*N + j)) * 2 + {0,1}]. */
void oracle_assemble_2d(int n, double h, double mu_t, int Lo, int Li,
                        const double *D, double *A)
{
    const long N = (long)n * n;
    const int Mo = 2 * Lo + 1, Mi = 2 * Li + 1;
    const long ncol = (long)Mi * N;
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        const int i1 = (int)(i % n), i2 = (int)(i / n);
        for (int ko = 0; ko < Mo; ++ko) {
            const int k = ko - Lo;
            double *row = A + ((long)ko * N + i) * ncol * 2;
            for (int ki = 0; ki < Mi; ++ki) {
                const int kp = ki - Li;
                for (long j = 0; j < N; ++j) {
                    const int j1 = (int)(j % n), j2 = (int)(j / n);
                    double e_re, e_im;
                    if (j == i) {
                        e_re = D[(kp - k) + Lo + Li];
                        e_im = 0.0;
                    } else {
                        const double d1 = (i1 - j1) * h, d2 = (i2 - j2) * h;
                        const double rr = sqrt(d1 * d1 + d2 * d2);
                        const double th = atan2(d2, d1);
                        const double w = h * h * kappa2(mu_t, rr);
                        e_re = w * cos((kp - k) * th);
                        e_im = w * sin((kp - k) * th);
                    }
                    row[((long)ki * N + j) * 2 + 0] = e_re;
                    row[((long)ki * N + j) * 2 + 1] = e_im;
                }
            }
        }
    }
}

void oracle_Ktilde_3d(int n, double h, double mu_t, double D,
                      const double *phi, double *out, const int *rows, int nrows)
{
    const long N = (long)n * n * n;
    const long nout = rows ? nrows : N;
    #pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < nout; ++r) {
        const long i = rows ? rows[r] : r;
        const int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
        double acc = 0.0;
        for (long j = 0; j < N; ++j) {
            if (j == i) {
                acc += D * phi[j];
                continue;
            }
            const int j1 = (int)(j % n), j2 = (int)((j / n) % n), j3 = (int)(j / ((long)n * n));
            const double d1 = (i1 - j1) * h, d2 = (i2 - j2) * h, d3 = (i3 - j3) * h;
            const double rr = sqrt(d1 * d1 + d2 * d2 + d3 * d3);
            acc += h * h * h * kappa3(mu_t, rr) * phi[j];
        }
        out[r] = acc;
    }
}

void oracle_assemble_3d(int n, double h, double mu_t, double D, double *A)
{
    const long N = (long)n * n * n;
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        const int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
        for (long j = 0; j < N; ++j) {
            if (j == i) { A[i * N + j] = D; continue; }
            const int j1 = (int)(j % n), j2 = (int)((j / n) % n), j3 = (int)(j / ((long)n * n));
            const double d1 = (i1 - j1) * h, d2 = (i2 - j2) * h, d3 = (i3 - j3) * h;
            const double rr = sqrt(d1 * d1 + d2 * d2 + d3 * d3);
            A[i * N + j] = h * h * h * kappa3(mu_t, rr);
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
