// Level-set advection through the phase-space Liouville equation (the hot loop).
//
// Sec. 4, Eqs. 16 and 19: the labels (position Y, angle vartheta) are constant along the
// bicharacteristics and tau grows at unit rate along them.  In pseudo-time on (x, z, theta):
//   d_t u = L(u) = -(Vx d_x u + Vz d_z u + thetadot d_theta u) + s_u,  s = 1 for tau, 0 otherwise,
// third-order HJ-WENO (Jiang & Peng) upwinded by the sign of each velocity component, Shu-Osher
// TVD-RK3 written in increment form
//   u1 = u + dt L(u);  u2 = u + 1/4 ((u1 - u) + dt L(u1));  u_new = u + 2/3 ((u2 - u) + dt L(u2)),
// which equals the convex-combination form.  tau is stored as a double-float pair and updated with
// an error-free sum, so the pseudo-time accumulation keeps ~48 significant bits without FP64
// arithmetic.  Angle-label differences are wrapped into [-pi, pi).  Frozen source-ball cells copy
// u^n; ghost layers are never written.
#include "egb_internal.cuh"

namespace egb {

struct StageArgs {
    Grid2D g;
    const float *uk;   // state being differentiated (u^n, u1 or u2)
    const float *un;   // u^n
    float *out;
    const float *Vx, *Vz, *Td;
    const int2 *ball;
    float dt, coef;    // coef = 1, 1/4, 2/3
    float ihx, ihz, idth;
    float eps[4];
};

// Third-order HJ-WENO one-sided derivative (undivided) from the differences d_{i-2} .. d_{i+1}.
// left: u^- from (d_{i-2}, d_{i-1}, d_i); right: u^+ from (d_{i-1}, d_i, d_{i+1}).
// With P the far difference, Q the near one and R the opposite one:
//   u = (d_{i-1} + d_i)/2 - w/2 (P - 2Q + R),  w = 1/(1 + 2 r^2),  r = (eps + (Q-P)^2)/(eps + (R-Q)^2)
// evaluated as w = B^2 / (B^2 + 2 A^2) with A = eps + (Q-P)^2, B = eps + (R-Q)^2.
__device__ __forceinline__ float weno3(float dm2, float dm1, float d0, float dp1, float eps, bool left) {
    float P = left ? dm2 : dp1;
    float Q = left ? dm1 : d0;
    float R = left ? d0 : dm1;
    float A = eps + (Q - P) * (Q - P);
    float B = eps + (R - Q) * (R - Q);
    float B2 = B * B;
    float w = B2 / (B2 + 2.f * A * A);
    return 0.5f * (dm1 + d0) - 0.5f * w * (P - 2.f * Q + R);
}

__device__ __forceinline__ float wrap_pi(float d) {
    const float two_pi = 6.28318530717958647692f;
    const float inv = 0.159154943091895335769f;
    return d - two_pi * rintf(d * inv);
}

// Derivative along one axis from 5 samples s[0..4] (cell at s[2]).
__device__ __forceinline__ float dir_deriv(const float s[5], float vel, float eps, bool angle) {
    float d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d[j] = s[j + 1] - s[j];
        if (angle) d[j] = wrap_pi(d[j]);
    }
    return weno3(d[0], d[1], d[2], d[3], eps, vel > 0.f);
}

__device__ __forceinline__ float dir_deriv_ff(const float h[5], const float l[5], float vel, float eps) {
    float d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = (h[j + 1] - h[j]) + (l[j + 1] - l[j]);
    return weno3(d[0], d[1], d[2], d[3], eps, vel > 0.f);
}

__global__ void __launch_bounds__(128) k_rk3_stage(StageArgs A) {
    const Grid2D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (ix >= g.nx || iz >= g.nz) return;
    int64_t p = pidx(g, k, iz, ix);
    int2 br = A.ball[iz];
    if (ix >= br.x && ix <= br.y) {
#pragma unroll
        for (int f = 0; f < NFIELD; ++f) A.out[f * g.field + p] = A.un[f * g.field + p];
        return;
    }
    int64_t c = cidx(g, k, iz, ix);
    float vx = __ldg(A.Vx + c), vz = __ldg(A.Vz + c), vt = __ldg(A.Td + c);
    int km2 = (k - 2 + g.nth) % g.nth, km1 = (k - 1 + g.nth) % g.nth;
    int kp1 = (k + 1) % g.nth, kp2 = (k + 2) % g.nth;
    int64_t off_t[5] = {(int64_t)(km2 - k) * g.plane, (int64_t)(km1 - k) * g.plane, 0,
                        (int64_t)(kp1 - k) * g.plane, (int64_t)(kp2 - k) * g.plane};
    float L[NFIELD - 1];
    float sx[5], sz[5], st[5], lx[5], lz[5], lt[5];
    // labels Yx, Yz, vartheta
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const float *u = A.uk + f * g.field + p;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            sx[m] = __ldg(u + (m - 2));
            sz[m] = __ldg(u + (int64_t)(m - 2) * g.pitch);
            st[m] = __ldg(u + off_t[m]);
        }
        bool ang = (f == 2);
        float ux = dir_deriv(sx, vx, A.eps[f], ang) * A.ihx;
        float uz = dir_deriv(sz, vz, A.eps[f], ang) * A.ihz;
        float ut = dir_deriv(st, vt, A.eps[f], ang) * A.idth;
        L[f] = -(vx * ux + vz * uz + vt * ut);
    }
    {  // tau as (hi, lo)
        const float *uh = A.uk + 3 * g.field + p;
        const float *ul = A.uk + 4 * g.field + p;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            sx[m] = __ldg(uh + (m - 2));
            lx[m] = __ldg(ul + (m - 2));
            sz[m] = __ldg(uh + (int64_t)(m - 2) * g.pitch);
            lz[m] = __ldg(ul + (int64_t)(m - 2) * g.pitch);
            st[m] = __ldg(uh + off_t[m]);
            lt[m] = __ldg(ul + off_t[m]);
        }
        float ux = dir_deriv_ff(sx, lx, vx, A.eps[3]) * A.ihx;
        float uz = dir_deriv_ff(sz, lz, vz, A.eps[3]) * A.ihz;
        float ut = dir_deriv_ff(st, lt, vt, A.eps[3]) * A.idth;
        L[3] = 1.f - (vx * ux + vz * uz + vt * ut);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        float un = __ldg(A.un + f * g.field + p);
        float uk = __ldg(A.uk + f * g.field + p);
        A.out[f * g.field + p] = un + A.coef * ((uk - un) + A.dt * L[f]);
    }
    {
        float hn = __ldg(A.un + 3 * g.field + p), ln = __ldg(A.un + 4 * g.field + p);
        float hk = __ldg(A.uk + 3 * g.field + p), lk = __ldg(A.uk + 4 * g.field + p);
        float inc = A.coef * (((hk - hn) + (lk - ln)) + A.dt * L[3]);
        ff r = ff_add_f(hn, ln, inc);
        A.out[3 * g.field + p] = r.hi;
        A.out[4 * g.field + p] = r.lo;
    }
}

cudaError_t launch_rk3_step(Solve &sv, float dt, cudaStream_t s) {
    const Grid2D &g = sv.g;
    StageArgs A;
    A.g = g;
    A.Vx = sv.vel;
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    A.Vz = sv.vel + cells;
    A.Td = sv.vel + 2 * cells;
    A.ball = sv.ball;
    A.dt = dt;
    A.ihx = (float)(1.0 / g.hx);
    A.ihz = (float)(1.0 / g.hz);
    A.idth = (float)(1.0 / g.dth);
    double h = g.hx > g.hz ? g.hx : g.hz;
    A.eps[0] = A.eps[1] = (float)(1e-6 * h * h);
    A.eps[2] = (float)(1e-6 * g.dth * g.dth);
    double cr = sv.c_ref;
    A.eps[3] = (float)(1e-6 * (h / cr) * (h / cr));
    dim3 block(32, 4);
    dim3 grid((g.nx + 31) / 32, (g.nz + 3) / 4, g.nth);
    int n = sv.cur, b1 = (sv.cur + 1) % 3, b2 = (sv.cur + 2) % 3;
    // stage 1: u1 = u + dt L(u)            -> buffer b1
    A.uk = sv.state[n]; A.un = sv.state[n]; A.out = sv.state[b1]; A.coef = 1.f;
    k_rk3_stage<<<grid, block, 0, s>>>(A);
    // stage 2: u2 = u + 1/4 ((u1-u) + dt L(u1)) -> buffer b2
    A.uk = sv.state[b1]; A.out = sv.state[b2]; A.coef = 0.25f;
    k_rk3_stage<<<grid, block, 0, s>>>(A);
    // stage 3: u_new = u + 2/3 ((u2-u) + dt L(u2)) -> buffer b1 (u1 no longer needed)
    A.uk = sv.state[b2]; A.out = sv.state[b1]; A.coef = 2.f / 3.f;
    k_rk3_stage<<<grid, block, 0, s>>>(A);
    sv.cur = b1;
    return cudaGetLastError();
}

}  // namespace egb
