/* Oracle (test infrastructure only): the 3-D TVD-RK3 / HJ-WENO3 level-set stepping of
 * liouville3d.py written out as plain float64 loops.
 *
 * Same scheme as liouville3d.py (Eqs. 16, 19 in pseudo-time on the phase space (x, y, z, th, ph)):
 *   L(u) = -(Vx u_x + Vy u_y + Vz u_z + thetadot u_th + phidot u_ph) + s_u, s = 1 for tau,
 *   L = 0 on frozen cells; ghosts (2 layers in x, y, z) keep their initial data; phi periodic;
 *   theta at cell centres, continued across a pole onto the opposite azimuth
 *   ((-th, ph) = (th, ph + pi), (pi + th, ph) = (pi - th, ph + pi)).
 *   Shu-Osher TVD-RK3, Jiang-Peng third-order HJ-WENO upwinded by the velocity sign.
 * Fields are padded arrays [nph][nth][nz+4][ny+4][nx+4] of doubles, x fastest; velocities and the
 * frozen mask are [nph][nth][nz][ny][nx].  Built with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define G3 2

static double weno3_side(double dm2, double dm1, double d0, double dp1, double eps, int left) {
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
    int nph, nth, nz, ny, nx, pz, py, px;
    double h[5]; /* hx, hy, hz, dth, dph */
    const double *vel[5]; /* Vx, Vy, Vz, thetadot, phidot */
    const unsigned char *frozen;
} grid3_t;

static size_t pidx3(const grid3_t *g, int k, int j, int iz, int iy, int ix) {
    return ((((size_t)k * g->nth + j) * g->pz + iz + G3) * g->py + iy + G3) * g->px + ix + G3;
}

/* padded index of the cell at angle offset m from (k, j) along phi (dim 4) or theta (dim 3) */
static size_t angle_neighbour(const grid3_t *g, int k, int j, int iz, int iy, int ix, int dim, int m) {
    if (dim == 4) {
        int kk = ((k + m) % g->nph + g->nph) % g->nph;
        return pidx3(g, kk, j, iz, iy, ix);
    }
    int jj = j + m, kk = k;
    if (jj < 0) { jj = -1 - jj; kk = (k + g->nph / 2) % g->nph; }
    else if (jj >= g->nth) { jj = 2 * g->nth - 1 - jj; kk = (k + g->nph / 2) % g->nph; }
    return pidx3(g, kk, jj, iz, iy, ix);
}

static double derivative3(const grid3_t *g, const double *u, int k, int j, int iz, int iy, int ix,
                          int dim, double vel, double eps) {
    double s[5];
    for (int m = -2; m <= 2; ++m) {
        size_t idx;
        if (dim == 0) idx = pidx3(g, k, j, iz, iy, ix + m);
        else if (dim == 1) idx = pidx3(g, k, j, iz, iy + m, ix);
        else if (dim == 2) idx = pidx3(g, k, j, iz + m, iy, ix);
        else idx = angle_neighbour(g, k, j, iz, iy, ix, dim, m);
        s[m + 2] = u[idx];
    }
    double d[4];
    for (int q = 0; q < 4; ++q) d[q] = s[q + 1] - s[q];
    return weno3_side(d[0], d[1], d[2], d[3], eps, vel > 0) / g->h[dim];
}

static void rhs3(const grid3_t *g, const double *u, double *L, double eps, double src) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nph; ++k)
        for (int j = 0; j < g->nth; ++j)
            for (int iz = 0; iz < g->nz; ++iz)
                for (int iy = 0; iy < g->ny; ++iy)
                    for (int ix = 0; ix < g->nx; ++ix) {
                        size_t c = ((((size_t)k * g->nth + j) * g->nz + iz) * g->ny + iy) * g->nx + ix;
                        if (g->frozen[c]) { L[c] = 0.0; continue; }
                        double acc = 0.0;
                        for (int dim = 0; dim < 5; ++dim) {
                            double v = g->vel[dim][c];
                            acc += v * derivative3(g, u, k, j, iz, iy, ix, dim, v, eps);
                        }
                        L[c] = -acc + src;
                    }
}

static void combine3(const grid3_t *g, double *w, const double *u, const double *v, const double *L,
                     double a, double b, double dt) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nph; ++k)
        for (int j = 0; j < g->nth; ++j)
            for (int iz = 0; iz < g->nz; ++iz)
                for (int iy = 0; iy < g->ny; ++iy)
                    for (int ix = 0; ix < g->nx; ++ix) {
                        size_t c = ((((size_t)k * g->nth + j) * g->nz + iz) * g->ny + iy) * g->nx + ix;
                        size_t p = pidx3(g, k, j, iz, iy, ix);
                        if (g->frozen[c]) { w[p] = u[p]; continue; }
                        w[p] = a * u[p] + b * (v[p] + dt * L[c]);
                    }
}

/* Advance the eight padded fields (bx, by, bz, n0x, n0y, n0z, q, tau) `steps` TVD-RK3 steps in
 * place.  eps[8]: WENO epsilon per field.  Returns 1 when the stage buffers cannot be allocated. */
int oracle3d_rk3_steps(int nph, int nth, int nz, int ny, int nx, double hx, double hy, double hz,
                       double dth, double dph, const double *Vx, const double *Vy, const double *Vz,
                       const double *Td, const double *Pd, const unsigned char *frozen,
                       const double *eps, double dt, int steps, double **fields) {
    grid3_t g = {nph, nth, nz, ny, nx, nz + 2 * G3, ny + 2 * G3, nx + 2 * G3,
                 {hx, hy, hz, dth, dph}, {Vx, Vy, Vz, Td, Pd}, frozen};
    size_t padded = (size_t)nph * nth * g.pz * g.py * g.px;
    size_t cells = (size_t)nph * nth * nz * ny * nx;
    double *u1 = malloc(padded * sizeof(double)), *u2 = malloc(padded * sizeof(double));
    double *L = malloc(cells * sizeof(double));
    if (!u1 || !u2 || !L) { free(u1); free(u2); free(L); return 1; }
    for (int s = 0; s < steps; ++s)
        for (int f = 0; f < 8; ++f) {
            double *u = fields[f];
            double src = (f == 7) ? 1.0 : 0.0;
            memcpy(u1, u, padded * sizeof(double));
            memcpy(u2, u, padded * sizeof(double));
            rhs3(&g, u, L, eps[f], src);
            combine3(&g, u1, u, u, L, 0.0, 1.0, dt);
            rhs3(&g, u1, L, eps[f], src);
            combine3(&g, u2, u, u1, L, 0.75, 0.25, dt);
            rhs3(&g, u2, L, eps[f], src);
            combine3(&g, u, u, u2, L, 1.0 / 3.0, 2.0 / 3.0, dt);
        }
    free(u1); free(u2); free(L);
    return 0;
}
