/* Direct O(N*M) summation u_i = sum_{j != i} G(x_i, x_j) q_j — oracle
 * (test infrastructure only; never linked into the library).
 *
 * This is the summation problem of Section 1, Eq. (1), with the Laplace
 * kernels of Eq. (2), the 3D Helmholtz kernel of Eq. (5) normalised as
 * e^{i kappa r} / (4 pi r), and the 2D Helmholtz kernel (i/4) H_0^(1)(kappa r)
 * = (i/4) (J_0 + i Y_0) with the C library's Bessel functions j0 / y0.
 * Coincident points (r == 0, which includes i == j) contribute nothing, like
 * the zero diagonal of A.
 *
 * Plain FP64 loops, OpenMP over targets, no blocking or reordering.
 *
 *   kind   0 = Laplace 2D, 1 = Laplace 3D, 2 = Helmholtz 3D, 3 = Helmholtz 2D
 *   xs     n x dim sources, row-major
 *   q      n x nrhs charges, each right-hand side contiguous; for Helmholtz
 *          interleaved complex (re, im) pairs
 *   xt     m x dim targets, row-major
 *   u      m x nrhs output, same layout as q (overwritten)
 */
#include <math.h>
#include <stdint.h>
#include <omp.h>

int oracle_num_threads(void) { return omp_get_max_threads(); }

void oracle_direct_sum(int kind, double kappa, int dim,
                       const double* xs, int64_t n,
                       const double* q, int nrhs,
                       const double* xt, int64_t m, double* u)
{
    const double four_pi = 4.0 * M_PI;
    const double two_pi = 2.0 * M_PI;
    const int cplx = (kind == 2 || kind == 3);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        for (int r = 0; r < nrhs; ++r) {
            double acc_re = 0.0, acc_im = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                double r2 = 0.0;
                for (int d = 0; d < dim; ++d) {
                    double t = xt[i * dim + d] - xs[j * dim + d];
                    r2 += t * t;
                }
                if (r2 == 0.0) continue;
                double dist = sqrt(r2);
                if (kind == 0) {
                    acc_re += (-log(dist) / two_pi) * q[(int64_t)r * n + j];
                } else if (kind == 1) {
                    acc_re += (1.0 / (four_pi * dist)) * q[(int64_t)r * n + j];
                } else {
                    double g_re, g_im;
                    if (kind == 2) {
                        g_re = cos(kappa * dist) / (four_pi * dist);
                        g_im = sin(kappa * dist) / (four_pi * dist);
                    } else {
                        g_re = -0.25 * y0(kappa * dist);
                        g_im = 0.25 * j0(kappa * dist);
                    }
                    double q_re = q[2 * ((int64_t)r * n + j)];
                    double q_im = q[2 * ((int64_t)r * n + j) + 1];
                    acc_re += g_re * q_re - g_im * q_im;
                    acc_im += g_re * q_im + g_im * q_re;
                }
            }
            if (cplx) {
                u[2 * ((int64_t)r * m + i)] = acc_re;
                u[2 * ((int64_t)r * m + i) + 1] = acc_im;
            } else {
                u[(int64_t)r * m + i] = acc_re;
            }
        }
    }
}
