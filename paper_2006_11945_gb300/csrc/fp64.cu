// The plain all-FP64 form of the evolution (comparison baseline).
//
// Same method and discretisation as the production path (Eq. 5 medium, Eqs. 3-12 velocities,
// Eq. 20 initial data, Eqs. 16/19 advected by HJ-WENO3 / TVD-RK3), written the straightforward way:
// every quantity in double precision, one thread per cell, neighbours read from global memory, one
// launch per RK stage, no TMA, no shared memory, no packing.  The one-pass superposition then reads
// the FP64 level sets through the production kernels after an exact conversion (labels rounded to
// FP32, tau split into a double-float pair).
#include "christoffel.cuh"

namespace egb {

__global__ void k_medium_a64(int nodes, const float *__restrict__ rho32, const float *__restrict__ c21,
                             double *__restrict__ a) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    double r = (double)rho32[n];
#pragma unroll
    for (int q = 0; q < 21; ++q) a[(int64_t)q * nodes + n] = (double)c21[(int64_t)n * 21 + q] / r;
}

__global__ void k_medium_grad64(int nx, int nz, double ihx, double ihz, const double *__restrict__ a,
                                double *__restrict__ dadx, double *__restrict__ dadz) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, q = blockIdx.z;
    if (ix >= nx) return;
    const double *f = a + (int64_t)q * nx * nz + (int64_t)iz * nx;
    double gx;
    if (ix == 0) gx = (4.0 * (f[1] - f[0]) - (f[2] - f[0])) * 0.5 * ihx;
    else if (ix == nx - 1) gx = (4.0 * (f[nx - 1] - f[nx - 2]) - (f[nx - 1] - f[nx - 3])) * 0.5 * ihx;
    else gx = (f[ix + 1] - f[ix - 1]) * 0.5 * ihx;
    const double *col = a + (int64_t)q * nx * nz + ix;
    double gz;
    if (iz == 0) gz = (4.0 * (col[nx] - col[0]) - (col[2 * nx] - col[0])) * 0.5 * ihz;
    else if (iz == nz - 1)
        gz = (4.0 * (col[(int64_t)(nz - 1) * nx] - col[(int64_t)(nz - 2) * nx]) -
              (col[(int64_t)(nz - 1) * nx] - col[(int64_t)(nz - 3) * nx])) * 0.5 * ihz;
    else gz = (col[(int64_t)(iz + 1) * nx] - col[(int64_t)(iz - 1) * nx]) * 0.5 * ihz;
    int64_t o = (int64_t)q * nx * nz + (int64_t)iz * nx + ix;
    dadx[o] = gx;
    dadz[o] = gz;
}

// Source slowness p_s(theta) in double (bilinear medium at x_s, as in the FP32 path).
__global__ void k_source64(const double *__restrict__ a, int nx, int nz, double ox, double oz, double hx,
                           double hz, double xs, double zs, int nth, double *ps) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nth) return;
    double fx = (xs - ox) / hx, fz = (zs - oz) / hz;
    int ix = (int)floor(fx), iz = (int)floor(fz);
    ix = ix < 0 ? 0 : (ix > nx - 2 ? nx - 2 : ix);
    iz = iz < 0 ? 0 : (iz > nz - 2 ? nz - 2 : iz);
    double tx = fx - ix, tz = fz - iz;
    int nodes = nx * nz, n00 = iz * nx + ix;
    double as[21];
    for (int q = 0; q < 21; ++q) {
        const double *f = a + (int64_t)q * nodes;
        as[q] = (1 - tz) * ((1 - tx) * f[n00] + tx * f[n00 + 1]) + tz * ((1 - tx) * f[n00 + nx] + tx * f[n00 + nx + 1]);
    }
    double th = 2.0 * M_PI * k / nth;
    double s = sin(th), c = cos(th);
    SrcVelT<double> r = source_velocity(as, s, c);
    ps[2 * k] = s / r.v;
    ps[2 * k + 1] = c / r.v;
}

__global__ void k_velocity64(int nx, int nz, int nth, const double *__restrict__ a,
                             const double *__restrict__ dadx, const double *__restrict__ dadz, Grid2D g,
                             double *__restrict__ velp, float *__restrict__ vel, float *rate_out) {
    int node = blockIdx.x * blockDim.x + threadIdx.x;
    int nodes = nx * nz;
    float rmax = 0.f;
    if (node < nodes) {
        double A[21], DX[21], DZ[21];
        for (int q = 0; q < 21; ++q) {
            A[q] = a[(int64_t)q * nodes + node];
            DX[q] = dadx[(int64_t)q * nodes + node];
            DZ[q] = dadz[(int64_t)q * nodes + node];
        }
        int64_t cells = (int64_t)nth * nodes;
        for (int k = 0; k < nth; ++k) {
            double th = 2.0 * M_PI * k / nth;
            RayVelT<double> r = ray_velocity2d(A, DX, DZ, sin(th), cos(th));
            int64_t o = (int64_t)k * nodes + node;
            vel[o] = (float)r.Vx;
            vel[cells + o] = (float)r.Vz;
            vel[2 * cells + o] = (float)r.td;
            vel[3 * cells + o] = (float)r.v;
            vel[4 * cells + o] = (float)r.pdx;
            vel[5 * cells + o] = (float)r.pdz;
            int64_t pp = pidx(g, k, node / nx, node % nx);
            velp[pp] = r.Vx;
            velp[g.field + pp] = r.Vz;
            velp[2 * g.field + pp] = r.td;
            double rate = fabs(r.Vx) / g.hx + fabs(r.Vz) / g.hz + fabs(r.td) / g.dth;
            rmax = fmaxf(rmax, (float)rate);
        }
    }
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

// Straight-ray data of the local medium on every padded cell (see the FP32 path).
__global__ void k_init64(Grid2D g, double xs, double zs, const double *__restrict__ velp,
                         const uint8_t *__restrict__ frozen, double *b0, double *b1, double *b2) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y, k = blockIdx.z;
    if (c >= g.pitch) return;
    int ix = c - XPAD, iz = r - ZPAD;
    int cx = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
    int cz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
    int64_t pc = pidx(g, k, cz, cx);
    double vx = velp[pc], vz = velp[g.field + pc];
    double th = 2.0 * M_PI * k / g.nth;
    double s = sin(th), cth = cos(th);
    double v = s * vx + cth * vz;  // n . V = v
    double x = g.ox + ix * g.hx - xs, z = g.oz + iz * g.hz - zs;
    double vn = sqrt(vx * vx + vz * vz);
    bool interior = ix >= 0 && ix < g.nx && iz >= 0 && iz < g.nz;
    double q = (interior && frozen[cidx(g, k, iz, ix)]) ? 1.0 : 0.0;
    double vals[4] = {(x * vz - z * vx) / vn, q, th, (s * x + cth * z) / v};
    int64_t o = (int64_t)k * g.plane + (int64_t)r * g.pitch + c;
    for (int f = 0; f < 4; ++f) {
        b0[f * g.field + o] = vals[f];
        b1[f * g.field + o] = vals[f];
        b2[f * g.field + o] = vals[f];
    }
}

__device__ __forceinline__ double weno3_64(double dm2, double dm1, double d0, double dp1, double eps, bool left) {
    double P = left ? dm2 : dp1, Q = left ? dm1 : d0, R = left ? d0 : dm1;
    double A = eps + (Q - P) * (Q - P);
    double B = eps + (R - Q) * (R - Q);
    double r = A / B;
    double w = 1.0 / (1.0 + 2.0 * r * r);
    return 0.5 * (dm1 + d0) - 0.5 * w * (P - 2.0 * Q + R);
}

__device__ __forceinline__ double wrap64(double d) {
    const double two_pi = 6.283185307179586476925286766559;
    return d - two_pi * rint(d / two_pi);
}

struct Stage64 {
    Grid2D g;
    const double *uk, *un;
    double *out;
    const double *V;  // padded [3]: Vx, Vz, thetadot (zero on frozen cells)
    double dt, coef, ihx, ihz, idth;
    double eps[4];
};

__global__ void k_rk3_stage64(Stage64 A) {
    const Grid2D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (ix >= g.nx || iz >= g.nz) return;
    int64_t p = pidx(g, k, iz, ix);
    double vx = A.V[p], vz = A.V[g.field + p], vt = A.V[2 * g.field + p];
    if (vx == 0.0 && vz == 0.0) {  // frozen cell of the source manifold
        for (int f = 0; f < 4; ++f) A.out[f * g.field + p] = A.un[f * g.field + p];
        return;
    }
    int kk[5] = {(k - 2 + g.nth) % g.nth, (k - 1 + g.nth) % g.nth, k, (k + 1) % g.nth, (k + 2) % g.nth};
    for (int f = 0; f < 4; ++f) {
        const double *u = A.uk + f * g.field;
        bool ang = (f == 2);
        double L = 0.0;
        for (int dir = 0; dir < 3; ++dir) {
            double s[5];
            for (int m = 0; m < 5; ++m) {
                int64_t q = dir == 0 ? p + (m - 2) : (dir == 1 ? p + (int64_t)(m - 2) * g.pitch
                                                               : pidx(g, kk[m], iz, ix));
                s[m] = u[q];
            }
            double d[4];
            for (int j = 0; j < 4; ++j) d[j] = ang ? wrap64(s[j + 1] - s[j]) : s[j + 1] - s[j];
            double vel = dir == 0 ? vx : (dir == 1 ? vz : vt);
            double ih = dir == 0 ? A.ihx : (dir == 1 ? A.ihz : A.idth);
            L -= vel * weno3_64(d[0], d[1], d[2], d[3], A.eps[f], vel > 0.0) * ih;
        }
        if (f == 3) L += 1.0;
        double un = A.un[f * g.field + p], uk = u[p];
        A.out[f * g.field + p] = un + A.coef * ((uk - un) + A.dt * L);
    }
}

__global__ void k_state64_to_32(Grid2D g, const double *__restrict__ s64, float *__restrict__ s32) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y, k = blockIdx.z;
    if (c >= g.pitch) return;
    int64_t o = (int64_t)k * g.plane + (int64_t)r * g.pitch + c;
    for (int f = 0; f < 3; ++f) s32[f * g.field + o] = (float)s64[f * g.field + o];
    double t = s64[3 * g.field + o];
    float hi = (float)t;
    s32[3 * g.field + o] = hi;
    s32[4 * g.field + o] = (float)(t - (double)hi);
}

__global__ void k_read_state64(Grid2D g, const double *__restrict__ st, double *out) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t p = pidx(g, k, iz, ix);
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    int64_t o = cidx(g, k, iz, ix);
    for (int f = 0; f < 4; ++f) out[f * cells + o] = st[f * g.field + p];
}

// ---- host side ------------------------------------------------------------------------------------
cudaError_t fp64_setup(Solve &sv, float *d_rate, cudaStream_t s) {
    const Grid2D &g = sv.g;
    const Medium &m = *sv.m;
    int nodes = g.nx * g.nz;
    double *a = nullptr, *dx = nullptr, *dz = nullptr, *ps = nullptr;
    cudaError_t e = cudaMalloc(&a, (size_t)nodes * 21 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dx, (size_t)nodes * 21 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dz, (size_t)nodes * 21 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&ps, (size_t)g.nth * 16);
    if (e == cudaSuccess) {
        // a = c / rho in double from the medium's copy of the FP32 inputs
        k_medium_a64<<<(nodes + 127) / 128, 128, 0, s>>>(nodes, m.rho, m.c21, a);
        dim3 grid((g.nx + 127) / 128, g.nz, 21);
        k_medium_grad64<<<grid, 128, 0, s>>>(g.nx, g.nz, 1.0 / g.hx, 1.0 / g.hz, a, dx, dz);
        k_source64<<<(g.nth + 127) / 128, 128, 0, s>>>(a, g.nx, g.nz, g.ox, g.oz, g.hx, g.hz, sv.xs, sv.zs,
                                                        g.nth, ps);
        k_velocity64<<<(nodes + 127) / 128, 128, 0, s>>>(g.nx, g.nz, g.nth, a, dx, dz, g, sv.velp64, sv.vel,
                                                         d_rate);
        dim3 gi((g.pitch + 127) / 128, g.nz + 2 * ZPAD, g.nth);
        e = launch_frozen_mask(sv, s);
        k_init64<<<gi, 128, 0, s>>>(g, sv.xs, sv.zs, sv.velp64, sv.frozen, sv.state64[0], sv.state64[1],
                                     sv.state64[2]);
        if (e == cudaSuccess) e = launch_zero_frozen_velocity(sv, s);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(a);
    cudaFree(dx);
    cudaFree(dz);
    cudaFree(ps);
    return e;
}

cudaError_t launch_rk3_step64(Solve &sv, double dt, cudaStream_t s) {
    const Grid2D &g = sv.g;
    Stage64 A;
    A.g = g;
    A.V = sv.velp64;
    A.dt = dt;
    A.ihx = 1.0 / g.hx;
    A.ihz = 1.0 / g.hz;
    A.idth = 1.0 / g.dth;
    double h = g.hx > g.hz ? g.hx : g.hz;
    A.eps[0] = 1e-6 * h * h;  // impact parameter (m)
    A.eps[1] = 1e-6;          // source indicator (dimensionless)
    A.eps[2] = 1e-6 * g.dth * g.dth;
    A.eps[3] = 1e-6 * (h / sv.c_ref) * (h / sv.c_ref);
    dim3 block(32, 4);
    dim3 grid((g.nx + 31) / 32, (g.nz + 3) / 4, g.nth);
    int n = sv.cur, b1 = (sv.cur + 1) % 3, b2 = (sv.cur + 2) % 3;
    A.un = sv.state64[n];
    A.uk = sv.state64[n]; A.out = sv.state64[b1]; A.coef = 1.0;
    k_rk3_stage64<<<grid, block, 0, s>>>(A);
    A.uk = sv.state64[b1]; A.out = sv.state64[b2]; A.coef = 0.25;
    k_rk3_stage64<<<grid, block, 0, s>>>(A);
    A.uk = sv.state64[b2]; A.out = sv.state64[b1]; A.coef = 2.0 / 3.0;
    k_rk3_stage64<<<grid, block, 0, s>>>(A);
    sv.cur = b1;
    return cudaGetLastError();
}

cudaError_t fp64_to_fp32_state(Solve &sv, cudaStream_t s) {
    const Grid2D &g = sv.g;
    dim3 gi((g.pitch + 127) / 128, g.nz + 2 * ZPAD, g.nth);
    k_state64_to_32<<<gi, 128, 0, s>>>(g, sv.state64[sv.cur], sv.state[0]);
    return cudaGetLastError();
}

cudaError_t launch_read_state64(const Solve &sv, double *out_dev, cudaStream_t s) {
    dim3 grid((sv.g.nx + 127) / 128, sv.g.nz, sv.g.nth);
    k_read_state64<<<grid, 128, 0, s>>>(sv.g, sv.state64[sv.cur], out_dev);
    return cudaGetLastError();
}

}  // namespace egb
