/*
 * FP64 CPU oracle for the source-to-waveform map.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this; the CUDA library never does.
 *
 * Everything here is a plain definition written out in double precision, with
 * no FFT, no blocking and no reordering of any sum:
 *
 *   bltt_apply      Eq. (time-domain-conv), Sec. II-C.2:
 *                     y_i[n] = sum_j sum_{k=0}^{n} f_ij[k] x_j[n-k]
 *                   which is also Eq. (elastic-response) with f = F_G, x = s
 *                   and Eq. (waveform-response) with f = F_q, x = v.
 *   dt_apply        v = D_t m, Sec. II-B.2: the backward difference
 *                     v[n] = (m[n] - m[n-1]) / dt,  m[-1] = 0.
 *   bltt_transpose  the transpose of bltt_apply (block upper-triangular
 *                   Toeplitz):  x_j[n] = sum_i sum_{k=0}^{Nt-1-n} f_ij[k] y_i[n+k]
 *   dt_transpose    the transpose of D_t:  u[n] = (w[n] - w[n+1]) / dt, w[Nt] = 0.
 *   dft_real        the DFT of a real sequence zero-padded to length L, bins
 *                   0..L/2 (Alg. 2, ZeroPad then FFT, written as the plain sum):
 *                     X[l] = sum_{n < n_in} x[n] exp(-2 pi i n l / L)
 *
 * Operators are row-major [Nout][Nin][Nt] (lag k fastest); signals are
 * [B][channels][Nt].  OpenMP splits only over independent output rows; each
 * output element is summed in the order of the formula above (j, then k), so
 * results do not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

/* y[b][i][n] = sum_j sum_{k<=n} F[i][j][k] * x[b][j][n-k].
 * The loop nest visits, for every fixed (b, i, n), the terms in the order
 * j = 0..Nin-1 and, within each j, k = 0..n: the order of the double sum. */
void oracle_bltt_apply(const double *F, long Nout, long Nin, int Nt,
                       const double *x, long B, double *y)
{
    long i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < Nout; ++i) {
        for (long b = 0; b < B; ++b) {
            double *yi = y + ((size_t)b * Nout + i) * Nt;
            memset(yi, 0, sizeof(double) * Nt);
            for (long j = 0; j < Nin; ++j) {
                const double *f = F + ((size_t)i * Nin + j) * Nt;
                const double *xj = x + ((size_t)b * Nin + j) * Nt;
                for (int k = 0; k < Nt; ++k) {
                    const double fk = f[k];
                    for (int n = k; n < Nt; ++n)
                        yi[n] += fk * xj[n - k];
                }
            }
        }
    }
}

/* x[b][j][n] = sum_i sum_{k<=Nt-1-n} F[i][j][k] * y[b][i][n+k]  (F^T y). */
void oracle_bltt_transpose(const double *F, long Nout, long Nin, int Nt,
                           const double *y, long B, double *x)
{
    long j;
#pragma omp parallel for schedule(dynamic, 1)
    for (j = 0; j < Nin; ++j) {
        for (long b = 0; b < B; ++b) {
            double *xj = x + ((size_t)b * Nin + j) * Nt;
            memset(xj, 0, sizeof(double) * Nt);
            for (long i = 0; i < Nout; ++i) {
                const double *f = F + ((size_t)i * Nin + j) * Nt;
                const double *yi = y + ((size_t)b * Nout + i) * Nt;
                for (int k = 0; k < Nt; ++k) {
                    const double fk = f[k];
                    for (int n = 0; n + k < Nt; ++n)
                        xj[n] += fk * yi[n + k];
                }
            }
        }
    }
}

/* v[r][n] = (m[r][n] - m[r][n-1]) / dt with m[r][-1] = 0, for rows r < R. */
void oracle_dt_apply(const double *m, long R, int Nt, double dt, double *v)
{
    for (long r = 0; r < R; ++r) {
        const double *mr = m + (size_t)r * Nt;
        double *vr = v + (size_t)r * Nt;
        for (int n = 0; n < Nt; ++n)
            vr[n] = (mr[n] - (n > 0 ? mr[n - 1] : 0.0)) / dt;
    }
}

/* u[r][n] = (w[r][n] - w[r][n+1]) / dt with w[r][Nt] = 0  (D_t^T w). */
void oracle_dt_transpose(const double *w, long R, int Nt, double dt, double *u)
{
    for (long r = 0; r < R; ++r) {
        const double *wr = w + (size_t)r * Nt;
        double *ur = u + (size_t)r * Nt;
        for (int n = 0; n < Nt; ++n)
            ur[n] = (wr[n] - (n + 1 < Nt ? wr[n + 1] : 0.0)) / dt;
    }
}

/* X[r][l] = sum_{n<n_in} x[r][n] exp(-2 pi i n l / L), l = 0..L/2. */
void oracle_dft_real(const double *x, long R, int n_in, int L,
                     double *Xre, double *Xim)
{
    const int nb = L / 2 + 1;
    long r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < R; ++r) {
        const double *xr = x + (size_t)r * n_in;
        for (int l = 0; l < nb; ++l) {
            double re = 0.0, im = 0.0;
            for (int n = 0; n < n_in; ++n) {
                /* reduce n*l modulo L before forming the angle */
                const double ang = 2.0 * M_PI * (double)(((long)n * l) % L) / L;
                re += xr[n] * cos(ang);
                im -= xr[n] * sin(ang);
            }
            Xre[(size_t)r * nb + l] = re;
            Xim[(size_t)r * nb + l] = im;
        }
    }
}
