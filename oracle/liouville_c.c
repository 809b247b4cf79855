/* Oracle (test infrastructure only): the TVD-RK3 / HJ-WENO3 level-set stepping of liouville.py
 * written out as plain float64 loops so that full 64x64x64 runs finish in seconds.
 *
 * Same scheme, same order of operations as liouville.py (Eqs. 16, 19, 20 of the paper in pseudo-time):
 *   L(u) = -(Vx u_x + Vz u_z + thetadot u_theta) + s_u, s = 1 for tau, 0 for the labels,
 *   L = 0 on frozen cells (the source manifold); ghosts (2 layers in x, z) keep their initial data;
 *   theta periodic; differences of the angle label wrapped into [-pi, pi).
 *   Shu-Osher TVD-RK3.  Jiang-Peng third-order HJ-WENO, upwinded by the velocity sign.
 * Fields are padded arrays [nth][nz+4][nx+4] of doubles, x fastest.
 * Built with -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define G 2

static double wrap_angle(double d) {
    const double two_pi = 6.283185307179586476925286766559;
    double r = fmod(d + M_PI, two_pi);
    if (r < 0) r += two_pi;
    return r - M_PI;
}

/* One-sided WENO3 derivative (undivided) from the differences d_{i-2}, d_{i-1}, d_i, d_{i+1}. */
static double weno3_upwind(double dm2, double dm1, double d0, double dp1, double eps, int left) {
    double centre = 0.5 * (dm1 + d0);
    if (left) {
        double a = dm1 - dm2, b = d0 - dm1;
        double r = (eps + a * a) / (eps + b * b);
        double w = 1.0 / (1.0 + 2.0 * r * r);
        return centre - 0.5 * w * (dm2 - 2.0 * dm1 + d0);
    } else {
        double a = dp1 - d0, b = d0 - dm1;
        double r = (eps + a * a) / (eps + b * b);
        double w = 1.0 / (1.0 + 2.0 * r * r);
        return centre - 0.5 * w * (dp1 - 2.0 * d0 + dm1);
    }
}

typedef struct {
    int nth, nz, nx, pz, px; /* pz = nz + 4, px = nx + 4 */
    double hx, hz, dth;
    const double *Vx, *Vz, *Td; /* [nth][nz][nx] */
    const unsigned char *ball;  /* [nth][nz][nx] frozen cells */
} grid_t;

static double derivative(const grid_t *g, const double *u, int k, int iz, int ix, int dim,
                         double vel, double eps, int angle) {
    double s[5];
    for (int m = -2; m <= 2; ++m) {
        size_t idx;
        if (dim == 0) idx = ((size_t)k * g->pz + iz + G) * g->px + ix + G + m;
        else if (dim == 1) idx = ((size_t)k * g->pz + iz + G + m) * g->px + ix + G;
        else {
            int kk = ((k + m) % g->nth + g->nth) % g->nth;
            idx = ((size_t)kk * g->pz + iz + G) * g->px + ix + G;
        }
        s[m + 2] = u[idx];
    }
    double d[4];
    for (int j = 0; j < 4; ++j) {
        d[j] = s[j + 1] - s[j];
        if (angle) d[j] = wrap_angle(d[j]);
    }
    double h = dim == 0 ? g->hx : (dim == 1 ? g->hz : g->dth);
    return weno3_upwind(d[0], d[1], d[2], d[3], eps, vel > 0) / h;
}

static void rhs(const grid_t *g, const double *u, double *L, double eps, int angle, double src) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nth; ++k)
        for (int iz = 0; iz < g->nz; ++iz)
            for (int ix = 0; ix < g->nx; ++ix) {
                size_t c = ((size_t)k * g->nz + iz) * g->nx + ix;
                if (g->ball[c]) { L[c] = 0.0; continue; }
                double vx = g->Vx[c], vz = g->Vz[c], vt = g->Td[c];
                double ux = derivative(g, u, k, iz, ix, 0, vx, eps, angle);
                double uz = derivative(g, u, k, iz, ix, 1, vz, eps, angle);
                double ut = derivative(g, u, k, iz, ix, 2, vt, eps, angle);
                L[c] = -(vx * ux + vz * uz + vt * ut) + src;
            }
}

/* w_interior = a * u + b * (v + dt * L); frozen cells copy u bit for bit */
static void combine(const grid_t *g, double *w, const double *u, const double *v, const double *L,
                    double a, double b, double dt) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nth; ++k)
        for (int iz = 0; iz < g->nz; ++iz)
            for (int ix = 0; ix < g->nx; ++ix) {
                size_t c = ((size_t)k * g->nz + iz) * g->nx + ix;
                size_t p = ((size_t)k * g->pz + iz + G) * g->px + ix + G;
                if (g->ball[c]) { w[p] = u[p]; continue; }
                w[p] = a * u[p] + b * (v[p] + dt * L[c]);
            }
}

/* Advance the four padded fields `steps` TVD-RK3 steps in place.  eps[4]: WENO epsilon per field. */
int oracle_rk3_steps(int nth, int nz, int nx, double hx, double hz, double dth,
                     const double *Vx, const double *Vz, const double *Td,
                     const unsigned char *ball, const double *eps, double dt, int steps,
                     double *b, double *q, double *Th, double *tau) {
    grid_t g = {nth, nz, nx, nz + 2 * G, nx + 2 * G, hx, hz, dth, Vx, Vz, Td, ball};
    size_t padded = (size_t)nth * g.pz * g.px, cells = (size_t)nth * nz * nx;
    double *fields[4] = {b, q, Th, tau};
    double *u1 = malloc(padded * sizeof(double)), *u2 = malloc(padded * sizeof(double));
    double *L = malloc(cells * sizeof(double));
    if (!u1 || !u2 || !L) { free(u1); free(u2); free(L); return 1; }
    for (int s = 0; s < steps; ++s)
        for (int f = 0; f < 4; ++f) {
            double *u = fields[f];
            int angle = (f == 2);
            double src = (f == 3) ? 1.0 : 0.0;
            memcpy(u1, u, padded * sizeof(double));
            memcpy(u2, u, padded * sizeof(double));
            rhs(&g, u, L, eps[f], angle, src);
            combine(&g, u1, u, u, L, 0.0, 1.0, dt);
            rhs(&g, u1, L, eps[f], angle, src);
            combine(&g, u2, u, u1, L, 0.75, 0.25, dt);
            rhs(&g, u2, L, eps[f], angle, src);
            combine(&g, u, u, u2, L, 1.0 / 3.0, 2.0 / 3.0, dt);
        }
    free(u1); free(u2); free(L);
    return 0;
}
