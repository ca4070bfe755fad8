/*
 * Seeded synthetic response operators (input generation only).
 *
 * This file builds the closed-form stand-ins for the precomputed impulse
 * responses of the paper (elastic Green's functions F_{G,k}, Sec. II-B.1;
 * acoustic-gravity adjoint responses F_{q,k}, Sec. II-B.2).  The real ones
 * come from FK and adjoint PDE solves that are out of reach here; these are
 * a decaying Ricker pulse delayed by the travel time:
 *
 *     out[a][b][k] = exp(-d_ab / decay) * ricker(k*dt - d_ab / vel; f0)
 *     ricker(tau; f0) = (1 - 2 pi^2 f0^2 tau^2) * exp(-pi^2 f0^2 tau^2)
 *
 * with d_ab the 3-D Euclidean distance (km) between point a of `pa` and
 * point b of `pb`.  It holds none of the method's arithmetic: it only fills
 * the operator arrays that both the FP64 oracle and the CUDA library are
 * given as inputs.
 */
#include <math.h>
#include <stddef.h>

static double ricker(double tau, double f0)
{
    const double a = M_PI * M_PI * f0 * f0 * tau * tau;
    return (1.0 - 2.0 * a) * exp(-a);
}

/* Fill out[a][b][k] for a < na, b < nb, k < Nt (row-major, k fastest).
 * pa: [na][3], pb: [nb][3] coordinates in km.  out_f32 != 0 writes float,
 * otherwise double.  Every value is computed in double. */
void synth_response(const double *pa, long na, const double *pb, long nb,
                    int Nt, double dt, double vel, double decay, double f0,
                    int out_f32, void *out)
{
    long a;
#pragma omp parallel for schedule(static)
    for (a = 0; a < na; ++a) {
        for (long b = 0; b < nb; ++b) {
            const double dx = pa[3 * a + 0] - pb[3 * b + 0];
            const double dy = pa[3 * a + 1] - pb[3 * b + 1];
            const double dz = pa[3 * a + 2] - pb[3 * b + 2];
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double amp = exp(-d / decay);
            const double delay = d / vel;
            const size_t base = ((size_t)a * (size_t)nb + (size_t)b) * (size_t)Nt;
            if (out_f32) {
                float *o = (float *)out + base;
                for (int k = 0; k < Nt; ++k)
                    o[k] = (float)(amp * ricker(k * dt - delay, f0));
            } else {
                double *o = (double *)out + base;
                for (int k = 0; k < Nt; ++k)
                    o[k] = amp * ricker(k * dt - delay, f0);
            }
        }
    }
}
