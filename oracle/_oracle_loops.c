/*
 * Oracle loops in plain C, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  These loops back the CPU oracle in oracle/*.py.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load this library; the CUDA product path never links,
 * loads or calls it, and shares no code with it.
 *
 * Conventions (the paper leaves the grid implicit; Sec. 2, Eq. (nonlocal53)):
 *   grid point x_{i,a} = (i_a - n_a/2) h_a, i_a = 0..n_a-1, C order, last axis
 *   fastest; d = 1, 2 or 3 (unused axes have n = 1 and contribute nothing).
 *   Complex arrays are interleaved (re, im) doubles.
 *
 * Fine-grid coordinates for the NUFFT are in units of fine cells: a node with
 * t = k h (radians) sits at z = t / (2 pi / nf).  The spreading function is the
 * "exponential of semicircle" (Barnett, Magland & af Klinteberg, SIAM J. Sci.
 * Comput. 41 (2019)):  phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), |z| < w/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

typedef int64_t i64;

/* thread control for timing the oracle on a stated number of host cores */
void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int orc_max_threads(void) { return omp_get_max_threads(); }

static void dims3(int d, const i64 *n, const double *h, i64 nn[3], double hh[3])
{
    for (int a = 0; a < 3; a++) {
        nn[a] = (a < d) ? n[a] : 1;
        hh[a] = (a < d && h) ? h[a] : 1.0;
    }
}

/*
 * Trapezoid Fourier transform at arbitrary nodes (the rho-hat of Eq. (ifft)
 * evaluated on the grid): out_j = (prod_a h_a) sum_i rho_i exp(-i k_j . x_i).
 * The sum is evaluated as nested 1D sums using exp(a+b+c) = exp(a)exp(b)exp(c).
 */
void orc_direct_type2(int d, const i64 *n, const double *h, const double *rho,
                      i64 M, const double *k, double *out)
{
    i64 nn[3];
    double hh[3];
    dims3(d, n, h, nn, hh);
    double vol = 1.0;
    for (int a = 0; a < d; a++) vol *= hh[a];
#pragma omp parallel
    {
        double *cs[3], *sn[3];
        for (int a = 0; a < 3; a++) {
            cs[a] = (double *)malloc(sizeof(double) * nn[a]);
            sn[a] = (double *)malloc(sizeof(double) * nn[a]);
        }
#pragma omp for schedule(dynamic, 16)
        for (i64 j = 0; j < M; j++) {
            for (int a = 0; a < 3; a++) {
                double ka = (a < d) ? k[j * d + a] : 0.0;
                for (i64 i = 0; i < nn[a]; i++) {
                    double x = (double)(i - nn[a] / 2) * hh[a];
                    cs[a][i] = cos(ka * x);
                    sn[a][i] = -sin(ka * x); /* exp(-i k x) = cos - i sin */
                }
            }
            double re = 0.0, im = 0.0;
            for (i64 i0 = 0; i0 < nn[0]; i0++) {
                double r0 = 0.0, m0 = 0.0;
                for (i64 i1 = 0; i1 < nn[1]; i1++) {
                    const double *row = rho + (i0 * nn[1] + i1) * nn[2];
                    double r1 = 0.0, m1 = 0.0;
                    for (i64 i2 = 0; i2 < nn[2]; i2++) {
                        r1 += row[i2] * cs[2][i2];
                        m1 += row[i2] * sn[2][i2];
                    }
                    r0 += r1 * cs[1][i1] - m1 * sn[1][i1];
                    m0 += r1 * sn[1][i1] + m1 * cs[1][i1];
                }
                re += r0 * cs[0][i0] - m0 * sn[0][i0];
                im += r0 * sn[0][i0] + m0 * cs[0][i0];
            }
            out[2 * j] = vol * re;
            out[2 * j + 1] = vol * im;
        }
        for (int a = 0; a < 3; a++) {
            free(cs[a]);
            free(sn[a]);
        }
    }
}

/*
 * Real part of the nonuniform-to-grid sum (the quadrature sum of Eq. (ifft)):
 * out_i = Re sum_j c_j exp(+i k_j . x_i)   for every grid point x_i.
 * Parallel over the first grid axis; per-node phase tables for axes 1 and 2.
 */
void orc_direct_type1(int d, const i64 *n, const double *h, i64 M, const double *k,
                      const double *c, double *out)
{
    i64 nn[3];
    double hh[3];
    dims3(d, n, h, nn, hh);
    i64 n12 = nn[1] + nn[2];
    double *T = (double *)malloc(sizeof(double) * 2 * (size_t)M * (size_t)n12);
#pragma omp parallel for schedule(static)
    for (i64 j = 0; j < M; j++) {
        double *t = T + 2 * j * n12;
        for (int a = 1; a < 3; a++) {
            double ka = (a < d) ? k[j * d + a] : 0.0;
            for (i64 i = 0; i < nn[a]; i++) {
                double x = (double)(i - nn[a] / 2) * hh[a];
                t[0] = cos(ka * x);
                t[1] = sin(ka * x);
                t += 2;
            }
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 i0 = 0; i0 < nn[0]; i0++) {
        double *acc = out + i0 * nn[1] * nn[2];
        memset(acc, 0, sizeof(double) * nn[1] * nn[2]);
        double x0 = (double)(i0 - nn[0] / 2) * hh[0];
        for (i64 j = 0; j < M; j++) {
            double a0 = k[j * d + 0] * x0;
            double e0r = cos(a0), e0i = sin(a0);
            double cr = c[2 * j], ci = c[2 * j + 1];
            double br = cr * e0r - ci * e0i, bi = cr * e0i + ci * e0r;
            const double *t1 = T + 2 * j * n12;
            const double *t2 = t1 + 2 * nn[1];
            for (i64 i1 = 0; i1 < nn[1]; i1++) {
                double er = br * t1[2 * i1] - bi * t1[2 * i1 + 1];
                double ei = br * t1[2 * i1 + 1] + bi * t1[2 * i1];
                double *row = acc + i1 * nn[2];
                for (i64 i2 = 0; i2 < nn[2]; i2++)
                    row[i2] += er * t2[2 * i2] - ei * t2[2 * i2 + 1];
            }
        }
    }
    free(T);
}

/* ---------------- plain NUFFT gridding (interpolate / spread) ---------------- */

static inline double es_phi(double z, int w, double beta)
{
    double x = 2.0 * z / (double)w;
    if (x <= -1.0 || x >= 1.0) return 0.0;
    return exp(beta * (sqrt(1.0 - x * x) - 1.0));
}

static inline i64 wrap(i64 l, i64 nf)
{
    i64 r = l % nf;
    return r < 0 ? r + nf : r;
}

/* first tap index and w kernel values of one node along one axis */
static void taps1d(double z, int w, double beta, i64 *l0, double *v)
{
    i64 s = (i64)ceil(z - 0.5 * (double)w);
    *l0 = s;
    for (int t = 0; t < w; t++) v[t] = es_phi((double)(s + t) - z, w, beta);
}

/*
 * Interpolation (body of the type-2 NUFFT):
 *   out_j = sum_l F_l prod_a phi(l_a - z_{j,a}),  l over the w^d fine points nearest
 *   z_j, indices taken mod nf (periodic fine grid).
 */
void orc_interp(int d, const i64 *nf, const double *F, i64 M, const double *z, int w,
                double beta, double *out)
{
    i64 nn[3];
    double hh[3];
    dims3(d, nf, NULL, nn, hh);
#pragma omp parallel for schedule(dynamic, 256)
    for (i64 j = 0; j < M; j++) {
        i64 l0[3] = {0, 0, 0};
        double v[3][64];
        int wa[3];
        for (int a = 0; a < 3; a++) {
            if (a < d) {
                wa[a] = w;
                taps1d(z[j * d + a], w, beta, &l0[a], v[a]);
            } else {
                wa[a] = 1;
                v[a][0] = 1.0;
            }
        }
        double re = 0.0, im = 0.0;
        for (int t0 = 0; t0 < wa[0]; t0++) {
            i64 p0 = wrap(l0[0] + t0, nn[0]);
            for (int t1 = 0; t1 < wa[1]; t1++) {
                i64 p1 = wrap(l0[1] + t1, nn[1]);
                double v01 = v[0][t0] * v[1][t1];
                for (int t2 = 0; t2 < wa[2]; t2++) {
                    i64 p2 = wrap(l0[2] + t2, nn[2]);
                    const double *f = F + 2 * ((p0 * nn[1] + p1) * nn[2] + p2);
                    double kv = v01 * v[2][t2];
                    re += kv * f[0];
                    im += kv * f[1];
                }
            }
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
}

/*
 * Spreading (body of the type-1 NUFFT):
 *   G_l += sum_j c_j prod_a phi(l_a - z_{j,a})   (periodic, G zeroed by the caller).
 * Each thread owns whole planes of the first axis; nodes are bucketed by their
 * first tap index along that axis so a plane visits exactly the nodes touching it.
 */
void orc_spread(int d, const i64 *nf, i64 M, const double *z, const double *c, int w,
                double beta, double *G)
{
    i64 nn[3];
    double hh[3];
    dims3(d, nf, NULL, nn, hh);
    /* counting sort of nodes by first-axis start tap (mod nf0) */
    i64 *cnt = (i64 *)calloc((size_t)nn[0] + 1, sizeof(i64));
    i64 *ord = (i64 *)malloc(sizeof(i64) * (size_t)(M > 0 ? M : 1));
    for (i64 j = 0; j < M; j++) {
        i64 s = (i64)ceil(z[j * d] - 0.5 * (double)w);
        cnt[wrap(s, nn[0]) + 1]++;
    }
    for (i64 b = 0; b < nn[0]; b++) cnt[b + 1] += cnt[b];
    i64 *pos = (i64 *)malloc(sizeof(i64) * (size_t)nn[0]);
    memcpy(pos, cnt, sizeof(i64) * (size_t)nn[0]);
    for (i64 j = 0; j < M; j++) {
        i64 s = (i64)ceil(z[j * d] - 0.5 * (double)w);
        ord[pos[wrap(s, nn[0])]++] = j;
    }
    free(pos);
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 p0 = 0; p0 < nn[0]; p0++) {
        double *plane = G + 2 * p0 * nn[1] * nn[2];
        for (int t0 = 0; t0 < w; t0++) {
            i64 b = wrap(p0 - t0, nn[0]);
            for (i64 q = cnt[b]; q < cnt[b + 1]; q++) {
                i64 j = ord[q];
                i64 l0[3] = {0, 0, 0};
                double v[3][64];
                int wa[3];
                for (int a = 0; a < 3; a++) {
                    if (a < d) {
                        wa[a] = w;
                        taps1d(z[j * d + a], w, beta, &l0[a], v[a]);
                    } else {
                        wa[a] = 1;
                        v[a][0] = 1.0;
                    }
                }
                double s0 = v[0][t0];
                double cr = c[2 * j] * s0, ci = c[2 * j + 1] * s0;
                for (int t1 = 0; t1 < wa[1]; t1++) {
                    i64 p1 = wrap(l0[1] + t1, nn[1]);
                    double br = cr * v[1][t1], bi = ci * v[1][t1];
                    for (int t2 = 0; t2 < wa[2]; t2++) {
                        i64 p2 = wrap(l0[2] + t2, nn[2]);
                        double *g = plane + 2 * (p1 * nn[2] + p2);
                        g[0] += br * v[2][t2];
                        g[1] += bi * v[2][t2];
                    }
                }
            }
        }
    }
    free(cnt);
    free(ord);
}
