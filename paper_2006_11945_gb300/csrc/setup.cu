// Medium preparation, characteristic velocities, source tables and initial level sets.
//
// Sec. 2, Eq. 5: a_ijkl = c_ijkl / rho (per node), with second-order central differences for its
// gradient (second-order one-sided at the grid edges) and a 6x6 Cholesky positive-definiteness
// check.  Eqs. 3-12: per phase cell the qP eigenpair and the ray velocities (christoffel.cuh).
// Eq. 20 generalised to the closest-approach manifold of the point source: straight-ray labels
// b = (x - x_s) x g, q, vartheta = theta, tau = p . (x - x_s) on every cell, ghosts included.
#include "christoffel.cuh"

namespace egb {

// ------------------------------- medium --------------------------------------------------------
__global__ void k_medium_a(int nodes, const float *__restrict__ c21, const float *__restrict__ rho,
                           float *__restrict__ a, unsigned *err) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    float r = rho[n];
    float c[21];
    bool ok = isfinite(r) && r > 0.f;
#pragma unroll
    for (int q = 0; q < 21; ++q) {
        c[q] = c21[(int64_t)n * 21 + q];
        ok = ok && isfinite(c[q]);
        a[(int64_t)q * nodes + n] = c[q] / r;
    }
    // Cholesky of the 6x6 Voigt matrix (scaled by its largest diagonal entry)
    float L[6][6];
    float sc = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) sc = fmaxf(sc, fabsf(c[tri21(i, i)]));
    sc = sc > 0.f ? 1.f / sc : 1.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float d = c[tri21(j, j)] * sc;
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        ok = ok && d > 0.f;
        float ljj = sqrtf(fmaxf(d, 1e-30f));
        L[j][j] = ljj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            float t = c[tri21(i, j)] * sc;
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / ljj;
        }
    }
    if (!ok) atomicOr(err, DeviceErrors::NOT_PD);
}

// Gradient of a = c / rho from the float inputs, evaluated in FP64 and rounded once: on fine grids
// the neighbour differences of FP32-rounded a would carry a relative error 2^-24 |a| / (h |grad a|).
__device__ __forceinline__ double a_at(const float *__restrict__ c21, const float *__restrict__ rho,
                                       int64_t node, int q) {
    return (double)c21[node * 21 + q] / (double)rho[node];
}

__global__ void k_medium_grad(int nx, int nz, double ihx, double ihz, const float *__restrict__ c21,
                              const float *__restrict__ rho, float *__restrict__ dadx,
                              float *__restrict__ dadz) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y;
    int q = blockIdx.z;
    if (ix >= nx) return;
    auto A = [&](int jx, int jz) { return a_at(c21, rho, (int64_t)jz * nx + jx, q); };
    double gx, gz;
    if (ix == 0) gx = (4.0 * (A(1, iz) - A(0, iz)) - (A(2, iz) - A(0, iz))) * 0.5 * ihx;
    else if (ix == nx - 1) gx = (4.0 * (A(nx - 1, iz) - A(nx - 2, iz)) - (A(nx - 1, iz) - A(nx - 3, iz))) * 0.5 * ihx;
    else gx = (A(ix + 1, iz) - A(ix - 1, iz)) * 0.5 * ihx;
    if (iz == 0) gz = (4.0 * (A(ix, 1) - A(ix, 0)) - (A(ix, 2) - A(ix, 0))) * 0.5 * ihz;
    else if (iz == nz - 1) gz = (4.0 * (A(ix, nz - 1) - A(ix, nz - 2)) - (A(ix, nz - 1) - A(ix, nz - 3))) * 0.5 * ihz;
    else gz = (A(ix, iz + 1) - A(ix, iz - 1)) * 0.5 * ihz;
    int64_t o = (int64_t)q * nx * nz + (int64_t)iz * nx + ix;
    dadx[o] = (float)gx;
    dadz[o] = (float)gz;
}

cudaError_t launch_medium_a(int nodes, const float *c21_dev, const float *rho_dev, float *a,
                            unsigned *d_err, cudaStream_t s) {
    k_medium_a<<<(nodes + 127) / 128, 128, 0, s>>>(nodes, c21_dev, rho_dev, a, d_err);
    return cudaGetLastError();
}

cudaError_t launch_medium_prep(const Medium &m, const float *c21_dev, const float *rho_dev,
                               unsigned *d_err, cudaStream_t s) {
    int nodes = m.nx * m.nz;
    k_medium_a<<<(nodes + 127) / 128, 128, 0, s>>>(nodes, c21_dev, rho_dev, m.a, d_err);
    dim3 grid((m.nx + 127) / 128, m.nz, 21);
    k_medium_grad<<<grid, 128, 0, s>>>(m.nx, m.nz, 1.0 / m.hx, 1.0 / m.hz, c21_dev, rho_dev, m.dadx,
                                       m.dadz);
    cudaMemcpyAsync(m.rho, rho_dev, sizeof(float) * nodes, cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

// ------------------------------- source block ---------------------------------------------------
// the source block's layout: src_ps, src_sc in egb_internal.cuh

__device__ void bilinear_weights(const Medium &m, double xs, double zs, int &ix, int &iz, double &tx,
                                 double &tz) {
    double fx = (xs - m.ox) / m.hx, fz = (zs - m.oz) / m.hz;
    ix = (int)floor(fx);
    iz = (int)floor(fz);
    ix = ix < 0 ? 0 : (ix > m.nx - 2 ? m.nx - 2 : ix);
    iz = iz < 0 ? 0 : (iz > m.nz - 2 ? m.nz - 2 : iz);
    tx = fx - ix;
    tz = fz - iz;
}

__global__ void k_source(Medium m, double xs, double zs, int nth, float *src) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int ix, iz;
    double tx, tz;
    bilinear_weights(m, xs, zs, ix, iz, tx, tz);
    int nodes = m.nx * m.nz;
    int n00 = iz * m.nx + ix;
    auto interp = [&](const float *f) {
        return (float)((1 - tz) * ((1 - tx) * f[n00] + tx * f[n00 + 1]) +
                       tz * ((1 - tx) * f[n00 + m.nx] + tx * f[n00 + m.nx + 1]));
    };
    float as[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) as[q] = interp(m.a + (int64_t)q * nodes);
    // near a qP-qS degeneracy (relative gap below QP_GAP_FP64): the source medium in FP64, the
    // moduli a = c / rho of the four nodes from the inputs, interpolated in double
    auto polished = [&](double sd, double cd) {
        double ad[21];
        for (int q = 0; q < 21; ++q) {
            auto A = [&](int n) { return (double)m.c21[(int64_t)n * 21 + q] / (double)m.rho[n]; };
            ad[q] = (1 - tz) * ((1 - tx) * A(n00) + tx * A(n00 + 1)) +
                    tz * ((1 - tx) * A(n00 + m.nx) + tx * A(n00 + m.nx + 1));
        }
        SrcVelT<double> r = source_velocity<double>(ad, sd, cd);
        return SrcVel{(float)r.v, (float)r.Vx, (float)r.Vz, (float)r.Vn};
    };
    if (k == 0) {
        for (int q = 0; q < 21; ++q) src[q] = as[q];
        src[21] = interp(m.rho);
        float gap0 = 1.f;
        SrcVel r0 = source_velocity(as, 0.f, 1.f, &gap0);
        if (!(gap0 >= QP_GAP_FP64)) r0 = polished(0.0, 1.0);
        src[22] = r0.v;
        src[23] = 0.f;
    }
    if (k >= nth) return;
    double th = 2.0 * M_PI * k / nth;
    float s = (float)sin(th), c = (float)cos(th);
    float gap = 1.f;
    SrcVel r = source_velocity(as, s, c, &gap);
    if (!(gap >= QP_GAP_FP64)) r = polished(sin(th), cos(th));
    src[src_ps(k)] = s / r.v;
    src[src_ps(k) + 1] = c / r.v;
    src[src_sc(nth, k)] = s;
    src[src_sc(nth, k) + 1] = c;
}

// ------------------------------- velocities ------------------------------------------------------
// One phase cell's ray velocities in FP64 from the input stiffness and density (a = c / rho exactly
// as the FP64 inputs give it), for cells whose qP eigenvalue lies within QP_GAP_FP64 of the next.
__device__ RayVel polished_velocity2d(const Medium &m, int node, const float *dx, const float *dz, int k, int nth) {
    double ad[21], dxd[21], dzd[21];
    const double rho = (double)m.rho[node];
#pragma unroll
    for (int q = 0; q < 21; ++q) {
        ad[q] = (double)m.c21[(int64_t)node * 21 + q] / rho;
        dxd[q] = (double)dx[q];
        dzd[q] = (double)dz[q];
    }
    const double th = 2.0 * M_PI * k / nth;
    RayVelT<double> r = ray_velocity2d<double>(ad, dxd, dzd, sin(th), cos(th));
    return RayVel{(float)r.v, (float)r.Vx, (float)r.Vz, (float)r.pdx, (float)r.pdz, (float)r.td};
}

// At most 128 registers (the FP32 loop needs about 100; the rarely taken FP64 polish would otherwise
// double the allocation and halve the resident warps of every launch).
__global__ void __launch_bounds__(128, 4) k_velocity(Medium m, Grid2D g, const float *__restrict__ src,
                                                     float *__restrict__ vel,
                           float *__restrict__ velp, float *rate_out) {
    int node = blockIdx.x * blockDim.x + threadIdx.x;
    int nodes = g.nx * g.nz;
    float rmax = 0.f;
    if (node < nodes) {
        float a[21], dx[21], dz[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) {
            a[q] = m.a[(int64_t)q * nodes + node];
            dx[q] = m.dadx[(int64_t)q * nodes + node];
            dz[q] = m.dadz[(int64_t)q * nodes + node];
        }
        int64_t cells = (int64_t)g.nth * nodes;
        float ihx = (float)(1.0 / g.hx), ihz = (float)(1.0 / g.hz), idth = (float)(1.0 / g.dth);
        for (int k = 0; k < g.nth; ++k) {
            float s = src[src_sc(g.nth, k)], c = src[src_sc(g.nth, k) + 1];
            float gap = 1.f;
            RayVel r = ray_velocity2d(a, dx, dz, s, c, &gap);
            if (!(gap >= QP_GAP_FP64)) r = polished_velocity2d(m, node, dx, dz, k, g.nth);
            int64_t o = (int64_t)k * nodes + node;
            vel[o] = r.Vx;
            vel[cells + o] = r.Vz;
            vel[2 * cells + o] = r.td;
            vel[3 * cells + o] = r.v;
            vel[4 * cells + o] = r.pdx;
            vel[5 * cells + o] = r.pdz;
            int64_t pp = pidx(g, k, node / g.nx, node % g.nx);
            velp[pp] = r.Vx;
            velp[g.field + pp] = r.Vz;
            velp[2 * g.field + pp] = r.td;
            rmax = fmaxf(rmax, fabsf(r.Vx) * ihx + fabsf(r.Vz) * ihz + fabsf(r.td) * idth);
        }
    }
    // block max -> one atomic per block (non-negative floats order like their bit patterns)
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    __shared__ float wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wmax[w]);
        atomicMax((int *)rate_out, __float_as_int(b));
    }
}

// Padded velocity copy (Vx, Vz, thetadot) of the TMA stencil from the stored velocities, for a
// solve that reuses the velocities of an earlier source on the same medium.
__global__ void k_velp_from_vel(Grid2D g, const float *__restrict__ vel, float *__restrict__ velp) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    int64_t o = cidx(g, k, iz, ix), pp = pidx(g, k, iz, ix);
    velp[pp] = vel[o];
    velp[g.field + pp] = vel[cells + o];
    velp[2 * g.field + pp] = vel[2 * cells + o];
}

cudaError_t launch_velp_from_vel(const Solve &sv, cudaStream_t s) {
    dim3 grid((sv.g.nx + 127) / 128, sv.g.nz, sv.g.nth);
    k_velp_from_vel<<<grid, 128, 0, s>>>(sv.g, sv.vel, sv.velp);
    return cudaGetLastError();
}

cudaError_t launch_source_block(const Solve &sv, cudaStream_t s) {
    k_source<<<(sv.g.nth + 127) / 128, 128, 0, s>>>(*sv.m, sv.xs, sv.zs, sv.g.nth, sv.src);
    return cudaGetLastError();
}

cudaError_t launch_solve_setup(const Solve &sv, unsigned *d_err, float *d_rate, cudaStream_t s) {
    (void)d_err;
    k_source<<<(sv.g.nth + 127) / 128, 128, 0, s>>>(*sv.m, sv.xs, sv.zs, sv.g.nth, sv.src);
    int nodes = sv.g.nx * sv.g.nz;
    k_velocity<<<(nodes + 127) / 128, 128, 0, s>>>(*sv.m, sv.g, sv.src, sv.vel, sv.velp, d_rate);
    return cudaGetLastError();
}

// ------------------------------- initial level sets ---------------------------------------------
// Straight-ray data of the local medium (media clamped to the nearest node for ghosts):
//   b = (x - x_s) x g,  q = 1 on the frozen source manifold else 0,  vartheta = theta,
//   tau = p . (x - x_s) with p = n / v.
__global__ void k_init(Grid2D g, double xs, double zs, const float *__restrict__ vel,
                       const uint8_t *__restrict__ frozen, float *b0, float *b1, float *b2) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    int k = blockIdx.z;
    __shared__ double sc[2];  // sin, cos of theta_k (one angle per block)
    if (threadIdx.x == 0) {
        double th = 2.0 * M_PI * k / g.nth;
        sc[0] = sin(th);
        sc[1] = cos(th);
    }
    __syncthreads();
    if (c >= g.pitch) return;
    int ix = c - XPAD, iz = r - ZPAD;
    int cx = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
    int cz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    int64_t o = cidx(g, k, cz, cx);
    float vx = vel[o], vz = vel[cells + o], v = vel[3 * cells + o];
    double x = g.ox + ix * g.hx - xs;
    double z = g.oz + iz * g.hz - zs;
    double th = 2.0 * M_PI * k / g.nth;
    double vn = sqrt((double)vx * vx + (double)vz * vz);
    double bb = (x * vz - z * vx) / vn;
    double tau = (sc[0] * x + sc[1] * z) / (double)v;
    bool interior = ix >= 0 && ix < g.nx && iz >= 0 && iz < g.nz;
    float q = (interior && frozen[cidx(g, k, iz, ix)]) ? 1.f : 0.f;
    float hi = (float)tau;
    float lo = (float)(tau - (double)hi);
    float vals[NFIELD] = {(float)bb, q, (float)th, hi, lo};
    int64_t p = (int64_t)k * g.plane + (int64_t)r * g.pitch + c;
#pragma unroll
    for (int f = 0; f < NFIELD; ++f) {
        b0[f * g.field + p] = vals[f];
        b1[f * g.field + p] = vals[f];
        b2[f * g.field + p] = vals[f];
    }
}

cudaError_t launch_init_state(const Solve &sv, cudaStream_t s) {
    dim3 grid((sv.g.pitch + 127) / 128, sv.g.nz + 2 * ZPAD, sv.g.nth);
    k_init<<<grid, 128, 0, s>>>(sv.g, sv.xs, sv.zs, sv.vel, sv.frozen, sv.state[0], sv.state[1], sv.state[2]);
    return cudaGetLastError();
}

// ------------------------------- frozen source manifold (FP64, once per solve) ----------------------
// Source-medium unit group direction g_s(theta_k) in double, a_s = c / rho interpolated bilinearly
// from the medium's copy of the inputs (as the oracle does): one thread per angle.
__global__ void k_source_dirs(Grid2D g, const float *__restrict__ c21, const float *__restrict__ rho,
                              double xs, double zs, double *__restrict__ gs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nth) return;
    double fx = (xs - g.ox) / g.hx, fz = (zs - g.oz) / g.hz;
    int jx = (int)floor(fx), jz = (int)floor(fz);
    jx = jx < 0 ? 0 : (jx > g.nx - 2 ? g.nx - 2 : jx);
    jz = jz < 0 ? 0 : (jz > g.nz - 2 ? g.nz - 2 : jz);
    double tx = fx - jx, tz = fz - jz;
    int n00 = jz * g.nx + jx;
    int nn[4] = {n00, n00 + 1, n00 + g.nx, n00 + g.nx + 1};
    double as[21];
    for (int q = 0; q < 21; ++q) {
        double f[4];
        for (int m = 0; m < 4; ++m) f[m] = (double)c21[(int64_t)nn[m] * 21 + q] / (double)rho[nn[m]];
        as[q] = (1 - tz) * ((1 - tx) * f[0] + tx * f[1]) + tz * ((1 - tx) * f[2] + tx * f[3]);
    }
    double th = 2.0 * M_PI * k / g.nth;
    SrcVelT<double> r = source_velocity(as, sin(th), cos(th));
    gs[2 * k] = r.Vx / r.Vn;
    gs[2 * k + 1] = r.Vz / r.Vn;
}

// Per cell: frozen = r^2 <= r0^2 || (r^2 <= R_Sigma^2 && (x - x_s) . g_s(theta_k) < 0), r = |x - x_s|,
// with every product and sum rounded separately so the decision is reproducible.
__global__ void k_frozen(Grid2D g, const double *__restrict__ gsd, double xs, double zs, double r0, double R,
                         uint8_t *__restrict__ frozen) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx) return;
    double gx = gsd[2 * k], gz = gsd[2 * k + 1];
    double dx = __dadd_rn(__dadd_rn(g.ox, __dmul_rn((double)ix, g.hx)), -xs);
    double dz = __dadd_rn(__dadd_rn(g.oz, __dmul_rn((double)iz, g.hz)), -zs);
    double r2 = __dadd_rn(__dmul_rn(dz, dz), __dmul_rn(dx, dx));
    double dot = __dadd_rn(__dmul_rn(dx, gx), __dmul_rn(dz, gz));
    // a cell on the closest-approach line (d . g_s at rounding level) belongs to the leaving half
    bool approach = dot < 0.0 && __dmul_rn(dot, dot) > __dmul_rn(1e-24, r2);
    bool f = r2 <= __dmul_rn(r0, r0) || (r2 <= __dmul_rn(R, R) && approach);
    frozen[cidx(g, k, iz, ix)] = f ? 1 : 0;
}

__global__ void k_zero_frozen(Grid2D g, const uint8_t *__restrict__ frozen, float *velp, double *velp64) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx || !frozen[cidx(g, k, iz, ix)]) return;
    int64_t p = pidx(g, k, iz, ix);
    for (int f = 0; f < 3; ++f) {
        if (velp) velp[f * g.field + p] = 0.f;
        if (velp64) velp64[f * g.field + p] = 0.0;
    }
}

cudaError_t launch_frozen_mask(const Solve &sv, cudaStream_t s) {
    k_source_dirs<<<(sv.g.nth + 127) / 128, 128, 0, s>>>(sv.g, sv.m->c21, sv.m->rho, sv.xs, sv.zs, sv.gs64);
    dim3 grid((sv.g.nx + 127) / 128, sv.g.nz, sv.g.nth);
    k_frozen<<<grid, 128, 0, s>>>(sv.g, sv.gs64, sv.xs, sv.zs, sv.r0, sv.R_sigma, sv.frozen);
    return cudaGetLastError();
}

cudaError_t launch_zero_frozen_velocity(const Solve &sv, cudaStream_t s) {
    dim3 grid((sv.g.nx + 127) / 128, sv.g.nz, sv.g.nth);
    k_zero_frozen<<<grid, 128, 0, s>>>(sv.g, sv.frozen, sv.velp, sv.velp64);
    return cudaGetLastError();
}

// ------------------------------- state read-back -------------------------------------------------
__global__ void k_read_state(Grid2D g, const float *__restrict__ st, double *out) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t p = pidx(g, k, iz, ix);
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    int64_t o = cidx(g, k, iz, ix);
    out[o] = st[p];
    out[cells + o] = st[g.field + p];
    out[2 * cells + o] = st[2 * g.field + p];
    out[3 * cells + o] = (double)st[3 * g.field + p] + (double)st[4 * g.field + p];
}

cudaError_t launch_read_state(const Solve &sv, double *out_dev, cudaStream_t s) {
    dim3 grid((sv.g.nx + 127) / 128, sv.g.nz, sv.g.nth);
    k_read_state<<<grid, 128, 0, s>>>(sv.g, sv.state[sv.cur], out_dev);
    return cudaGetLastError();
}

}  // namespace egb
