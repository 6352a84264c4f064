/*
 * Oracle direct sums (test infrastructure only: imported by the tests, the
 * smoke check and the benchmark's CPU-baseline leg; never by the library).
 *
 * Plain FP64 double loops, one target at a time, OpenMP over targets.  Each
 * pair is evaluated from the kernel's definition as printed in Sec. 2
 * (Eqs. oseen, stresslet); no blocking, no reordering beyond the sum order.
 *
 *   Stokeslet  G(r) = (I + rhat rhat) / (8 pi mu |r|)                  Eq. oseen
 *   Stresslet  T_abc(r) = -(3 / 4 pi) rhat_a rhat_b rhat_c / |r|^2       Eq. stresslet
 *              (the 1/mu factor is dropped so that the double layer of a
 *               constant density is that constant inside the surface)
 *   r = target - source, n = outward normal of the source surface.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* u_i = sum_j G(x_i - y_j) wf_j over all sources j, skipping pairs with
 * tgt_fiber[i] == src_fiber[j] when both id arrays are given
 * (complementary fiber velocity, Eq. complementary-uf). */
void oracle_stokeslet(int64_t n_tgt, const double *tgt, const int32_t *tgt_fiber,
                      int64_t n_src, const double *src, const int32_t *src_fiber,
                      const double *wf, double mu, double *out)
{
    const double c = 1.0 / (8.0 * M_PI * mu);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_tgt; ++i) {
        double u0 = 0.0, u1 = 0.0, u2 = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            if (tgt_fiber && src_fiber && tgt_fiber[i] == src_fiber[j]) continue;
            double r0 = tgt[3 * i + 0] - src[3 * j + 0];
            double r1 = tgt[3 * i + 1] - src[3 * j + 1];
            double r2 = tgt[3 * i + 2] - src[3 * j + 2];
            double rn = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            double h0 = r0 / rn, h1 = r1 / rn, h2 = r2 / rn;
            const double *f = wf + 3 * j;
            double hf = h0 * f[0] + h1 * f[1] + h2 * f[2];
            u0 += c * (f[0] + h0 * hf) / rn;
            u1 += c * (f[1] + h1 * hf) / rn;
            u2 += c * (f[2] + h2 * hf) / rn;
        }
        out[3 * i + 0] = u0;
        out[3 * i + 1] = u1;
        out[3 * i + 2] = u2;
    }
}

/* u_i = sum_j w_j T(x_i - y_j) : (q_j n_j) -- the double-layer potential
 * of Eq. double-layer at targets off the surface (Eq. cortex-vel). */
void oracle_stresslet(int64_t n_tgt, const double *tgt, int64_t n_src, const double *src,
                      const double *normal, const double *w, const double *q, double *out)
{
    const double c = -3.0 / (4.0 * M_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_tgt; ++i) {
        double u[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n_src; ++j) {
            double r[3], h[3];
            for (int a = 0; a < 3; ++a) r[a] = tgt[3 * i + a] - src[3 * j + a];
            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int a = 0; a < 3; ++a) h[a] = r[a] / rn;
            /* T_abc q_b n_c, written as the triple contraction */
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int b = 0; b < 3; ++b)
                    for (int cc = 0; cc < 3; ++cc)
                        s += c * h[a] * h[b] * h[cc] / (rn * rn) * q[3 * j + b] * normal[3 * j + cc];
                u[a] += w[j] * s;
            }
        }
        for (int a = 0; a < 3; ++a) out[3 * i + a] = u[a];
    }
}

/* On-surface operator of the periphery equation (Eq. main-cortex-density)
 * with singularity subtraction (Sec. 3.1.2).  The fluid lies inside the
 * periphery and n points out of it, so the limit of T[q] from the fluid side
 * is q/2 + T_pv[q] (T[c] = c inside, c/2 on S); with T_pv[q](y_i) =
 * T_pv[q - q_i](y_i) + q_i/2:
 *   out_i = sum_{j != i} w_j T(y_i - y_j) : ((q_j - q_i) n_j) + q_i
 *         + n_i sum_j w_j (n_j . q_j)                       (rank completion N)
 * which equals q_i/2 + T_pv[q](y_i) + N[q](y_i). */
void oracle_surface_self(int64_t n, const double *y, const double *normal, const double *w,
                         const double *q, double *out)
{
    const double c = -3.0 / (4.0 * M_PI);
    double nq = 0.0;
    for (int64_t j = 0; j < n; ++j)
        nq += w[j] * (normal[3 * j] * q[3 * j] + normal[3 * j + 1] * q[3 * j + 1] +
                      normal[3 * j + 2] * q[3 * j + 2]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double u[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3], h[3], dq[3];
            for (int a = 0; a < 3; ++a) r[a] = y[3 * i + a] - y[3 * j + a];
            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int a = 0; a < 3; ++a) {
                h[a] = r[a] / rn;
                dq[a] = q[3 * j + a] - q[3 * i + a];
            }
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int b = 0; b < 3; ++b)
                    for (int cc = 0; cc < 3; ++cc)
                        s += c * h[a] * h[b] * h[cc] / (rn * rn) * dq[b] * normal[3 * j + cc];
                u[a] += w[j] * s;
            }
        }
        for (int a = 0; a < 3; ++a) out[3 * i + a] = u[a] + q[3 * i + a] + normal[3 * i + a] * nq;
    }
}

/* Diagonal of the on-surface operator above (periphery Jacobi entries of
 * Eq. prec): coefficient of q_{i,a} in row (i,a). */
void oracle_surface_diag(int64_t n, const double *y, const double *normal, const double *w,
                         double *out)
{
    const double c = -3.0 / (4.0 * M_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double r[3], h[3];
                for (int b = 0; b < 3; ++b) r[b] = y[3 * i + b] - y[3 * j + b];
                double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                for (int b = 0; b < 3; ++b) h[b] = r[b] / rn;
                double t = 0.0;
                for (int cc = 0; cc < 3; ++cc) t += c * h[a] * h[a] * h[cc] / (rn * rn) * normal[3 * j + cc];
                s -= w[j] * t;
            }
            out[3 * i + a] = s + 1.0 + w[i] * normal[3 * i + a] * normal[3 * i + a];
        }
    }
}

/* Rigid body surface, fluid OUTSIDE (Eq. main-nsb-second-kind): the limit of
 * the double layer from the fluid side is -q/2 + T_pv[q]; with the Gauss
 * identity (the double layer of a constant c is 0 outside, c/2 on the
 * surface) it is the subtracted sum
 *   out_i = sum_{j != i} w_j T(y_i - y_j) : ((q_j - q_i) n_j).
 * No rank completion here: the body's Stokeslet, rotlet and rigid-motion
 * unknowns are added by the caller. */
void oracle_body_self(int64_t n, const double *y, const double *normal, const double *w,
                      const double *q, double *out)
{
    const double c = -3.0 / (4.0 * M_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double u[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3], h[3], dq[3];
            for (int a = 0; a < 3; ++a) r[a] = y[3 * i + a] - y[3 * j + a];
            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int a = 0; a < 3; ++a) {
                h[a] = r[a] / rn;
                dq[a] = q[3 * j + a] - q[3 * i + a];
            }
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int b = 0; b < 3; ++b)
                    for (int cc = 0; cc < 3; ++cc)
                        s += c * h[a] * h[b] * h[cc] / (rn * rn) * dq[b] * normal[3 * j + cc];
                u[a] += w[j] * s;
            }
        }
        for (int a = 0; a < 3; ++a) out[3 * i + a] = u[a];
    }
}

/* Diagonal of oracle_body_self: coefficient of q_{i,a} in row (i,a)
 * (Jacobi entries of the body block, Eq. prec). */
void oracle_body_diag(int64_t n, const double *y, const double *normal, const double *w,
                      double *out)
{
    const double c = -3.0 / (4.0 * M_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double r[3], h[3];
                for (int b = 0; b < 3; ++b) r[b] = y[3 * i + b] - y[3 * j + b];
                double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                for (int b = 0; b < 3; ++b) h[b] = r[b] / rn;
                double t = 0.0;
                for (int cc = 0; cc < 3; ++cc) t += c * h[a] * h[a] * h[cc] / (rn * rn) * normal[3 * j + cc];
                s -= w[j] * t;
            }
            out[3 * i + a] = s;
        }
    }
}
