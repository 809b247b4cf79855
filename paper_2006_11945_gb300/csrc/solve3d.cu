// 3-D path: 5-D phase space (x, y, z, theta, phi).
//
// Sec. 2-5 in three dimensions.  Eqs. 3-12 with the full direction n = (sin th cos ph,
// sin th sin ph, cos th): V = a p g g, dp/dt = -1/2 g Gamma(grad a, p) g, and the direction angles
// move as dth/dt = v n_th . dp/dt, dph/dt = v e_ph . dp/dt / sin th.  Labels (Eqs. 16, 19 in
// pseudo-time): b (3-vector offset of the ray from x_s at closest approach; b = 0 is Eq. 35's
// Gamma), n0 (take-off phase direction), q (source indicator), tau (double-float).  Eq. 20's
// initial surface is the closest-approach manifold of the point source: cells within r0 of x_s, or
// within R_Sigma while their ray still approaches the source, hold straight-ray data forever.
//
//  k_medium_grad3d  grad a in FP64 from the float inputs (second order, one-sided at edges)
//  k_source3d       a_s, rho_s, c_ref and the FP64 unit group direction of every direction cell
//  k_velocity3d     per node, every direction: V, dp/dt, thetadot, phidot, v; CFL rate maximum
//  k_frozen3d       FP64 frozen-manifold decision (fixed rounding order)
//  k_init3d         straight-ray labels on every padded cell
//  k_rk3_3d<S>      one Shu-Osher stage: HJ-WENO3 upwind in all five dimensions, two x-neighbours
//                   per thread in packed FP32x2, theta continued across the poles, phi periodic
//  k_arrivals3d     per node: zeros of b over the (theta, phi) sphere -> T and |u| per arrival
//  k_centres3d      per direction cell and grid plane: zeros of b in the plane (beam centres)
//  k_beam3d         per centre: dynamic ray tracing from the label gradients (FP64 algebra) ->
//                   complex Hessian, spreading, amplitude, weight, exp(i omega tau)
//  k_sum3d          per receiver: the beams centred in its three grid planes (Eq. 34)
#include "christoffel.cuh"

namespace egb {

namespace s3 {

constexpr int KC3 = 4;  // beam centres kept per (plane, direction cell)

// ---- packed two-cell arithmetic --------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Upwind side of two cells along one axis: flow towards + (left-biased stencil) or towards -.
struct Up2 {
    bool lx, ly;
    float2 sig;  // +1 towards +, -1 otherwise
};
__device__ __forceinline__ Up2 upwind2(float2 v) {
    Up2 u;
    u.lx = v.x > 0.f;
    u.ly = v.y > 0.f;
    u.sig = f2(u.lx ? 1.f : -1.f, u.ly ? 1.f : -1.f);
    return u;
}

// Jiang-Peng HJ-WENO3 one-sided derivative of two cells from the differences d_j = s_{j+1} - s_j
// of their 5-point stencils, in second-difference form: with e_j = d_{j+1} - d_j, e_up = e_0
// (flow towards +) or e_2 (towards -), A = e_up^2 + eps, B = e_1^2 + eps and the weight
// w = 1 / (1 + 2 (A/B)^2) = B^2 / (B^2 + 2 A^2),
//     2 h u_x = (d_1 + d_2) + sig w (e_up - e_1)
// (the central difference less w/2 times the upwind curvature).  Returns 2 h u_x.
__device__ __forceinline__ float2 weno(const float2 d[4], const Up2 &up, float2 eps2) {
    float2 e0 = sub2(d[1], d[0]), e1 = sub2(d[2], d[1]), e2 = sub2(d[3], d[2]);
    float2 E = f2(up.lx ? e0.x : e2.x, up.ly ? e0.y : e2.y);
    float2 A = fma2(E, E, eps2);
    float2 B = fma2(e1, e1, eps2);
    float2 B2 = mul2(B, B);
    float2 den = fma2(mul2(A, A), f2(2.f, 2.f), B2);
    float2 num = mul2(B2, up.sig);
    float2 w = f2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    return fma2(w, sub2(E, e1), add2(d[1], d[2]));
}

__device__ __forceinline__ float2 deriv(const float2 s[5], const Up2 &up, float2 eps2) {
    float2 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = sub2(s[j + 1], s[j]);
    return weno(d, up, eps2);
}

__device__ __forceinline__ float2 deriv_ff(const float2 h[5], const float2 l[5], const Up2 &up, float2 eps2) {
    float2 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = add2(sub2(h[j + 1], h[j]), sub2(l[j + 1], l[j]));
    return weno(d, up, eps2);
}

// direction cell reached from (k, j) by m steps in theta, continued across the poles
__device__ __forceinline__ int theta_neighbour(const Grid3D &g, int k, int j, int m) {
    int jj = j + m, kk = k;
    if (jj < 0) { jj = -1 - jj; kk = (k + g.nph / 2) % g.nph; }
    else if (jj >= g.nth) { jj = 2 * g.nth - 1 - jj; kk = (k + g.nph / 2) % g.nph; }
    return kk * g.nth + jj;
}

__device__ __forceinline__ int phi_neighbour(const Grid3D &g, int k, int j, int m) {
    int kk = ((k + m) % g.nph + g.nph) % g.nph;
    return kk * g.nth + j;
}

// Orthonormal (e1, e2) perpendicular to the unit vector u: a = the axis with the smallest |u_a|
// (the first on ties), e1 = (E_a - u_a u)/|.|, e2 = u x e1.
template <typename R>
__device__ __forceinline__ void frame(const R u[3], R e1[3], R e2[3]) {
    int a = 0;
    R m = fabs(u[0]);
    if (fabs(u[1]) < m) { a = 1; m = fabs(u[1]); }
    if (fabs(u[2]) < m) { a = 2; }
    R ua = u[a];
    for (int i = 0; i < 3; ++i) e1[i] = (i == a ? R(1) : R(0)) - ua * u[i];
    R inv = R(1) / sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] *= inv;
    e2[0] = u[1] * e1[2] - u[2] * e1[1];
    e2[1] = u[2] * e1[0] - u[0] * e1[2];
    e2[2] = u[0] * e1[1] - u[1] * e1[0];
}

// a x b rounded term by term (no fused multiply-add), so that cross2(a, b) == -cross2(b, a) exactly:
// the two triangles sharing an edge then see opposite edge functions and a point on the edge is
// claimed by exactly one of them
__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) {
    return __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
}

// edge function cross(Pa, Pb) with a zero decided by the lexicographic sign of Pb - Pa
__device__ __forceinline__ float edge_sign(float ax, float ay, float bx, float by) {
    float E = cross2(ax, ay, bx, by);
    if (E > 0.f) return 1.f;
    if (E < 0.f) return -1.f;
    float dx = bx - ax, dy = by - ay;
    return (dx > 0.f || (dx == 0.f && dy > 0.f)) ? 1.f : -1.f;
}

// origin in the triangle (P0, P1, P2) of projected values; barycentric weights on success
__device__ __forceinline__ bool origin_in(const float P[3][2], float w[3]) {
    float area = cross2(P[1][0] - P[0][0], P[1][1] - P[0][1], P[2][0] - P[0][0], P[2][1] - P[0][1]);
    if (area == 0.f) return false;
    float sa = area > 0.f ? 1.f : -1.f;
    if (edge_sign(P[0][0], P[0][1], P[1][0], P[1][1]) != sa) return false;
    if (edge_sign(P[1][0], P[1][1], P[2][0], P[2][1]) != sa) return false;
    if (edge_sign(P[2][0], P[2][1], P[0][0], P[0][1]) != sa) return false;
    w[0] = cross2(P[1][0], P[1][1], P[2][0], P[2][1]) / area;
    w[1] = cross2(P[2][0], P[2][1], P[0][0], P[0][1]) / area;
    w[2] = cross2(P[0][0], P[0][1], P[1][0], P[1][1]) / area;
    return true;
}

}  // namespace s3

using namespace s3;

// ------------------------------- medium --------------------------------------------------------
__device__ __forceinline__ double a_node(const float *__restrict__ c21, const float *__restrict__ rho,
                                         int64_t node, int q) {
    return (double)c21[node * 21 + q] / (double)rho[node];
}

__global__ void k_medium_grad3d(int nx, int ny, int nz, double ihx, double ihy, double ihz,
                                const float *__restrict__ c21, const float *__restrict__ rho,
                                float *__restrict__ dadx, float *__restrict__ dady, float *__restrict__ dadz) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y % ny, iz = blockIdx.y / ny, q = blockIdx.z;
    if (ix >= nx) return;
    auto A = [&](int jx, int jy, int jz) { return a_node(c21, rho, ((int64_t)jz * ny + jy) * nx + jx, q); };
    auto d = [&](int i, int n, double ih, auto F) {
        if (i == 0) return (4.0 * (F(1) - F(0)) - (F(2) - F(0))) * 0.5 * ih;
        if (i == n - 1) return (4.0 * (F(n - 1) - F(n - 2)) - (F(n - 1) - F(n - 3))) * 0.5 * ih;
        return (F(i + 1) - F(i - 1)) * 0.5 * ih;
    };
    double gx = d(ix, nx, ihx, [&](int m) { return A(m, iy, iz); });
    double gy = d(iy, ny, ihy, [&](int m) { return A(ix, m, iz); });
    double gz = d(iz, nz, ihz, [&](int m) { return A(ix, iy, m); });
    int64_t o = (int64_t)q * nx * ny * nz + ((int64_t)iz * ny + iy) * nx + ix;
    dadx[o] = (float)gx;
    dady[o] = (float)gy;
    dadz[o] = (float)gz;
}

cudaError_t launch_medium_prep3d(const Medium &m, const float *c21_dev, const float *rho_dev,
                                 unsigned *d_err, cudaStream_t s) {
    int nodes = m.nx * m.ny * m.nz;
    cudaError_t e = launch_medium_a(nodes, c21_dev, rho_dev, m.a, d_err, s);
    if (e != cudaSuccess) return e;
    dim3 grid((m.nx + 127) / 128, m.ny * m.nz, 21);
    k_medium_grad3d<<<grid, 128, 0, s>>>(m.nx, m.ny, m.nz, 1.0 / m.hx, 1.0 / m.hy, 1.0 / m.hz, c21_dev,
                                         rho_dev, m.dadx, m.dady, m.dadz);
    cudaMemcpyAsync(m.rho, rho_dev, sizeof(float) * nodes, cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

// ------------------------------- source --------------------------------------------------------
// a_s = c / rho and rho at x_s by trilinear interpolation in FP64 (weights (wx wy) wz, summed over
// dz, dy, dx in that order).
__device__ void source_moduli(const Grid3D &g, const float *c21, const float *rho, double xs, double ys,
                              double zs, double as[21], double &rho_s) {
    double f[3] = {(xs - g.ox) / g.hx, (ys - g.oy) / g.hy, (zs - g.oz) / g.hz};
    int n[3] = {g.nx, g.ny, g.nz};
    int i[3];
    double t[3];
    for (int d = 0; d < 3; ++d) {
        int c = (int)floor(f[d]);
        c = c < 0 ? 0 : (c > n[d] - 2 ? n[d] - 2 : c);
        i[d] = c;
        t[d] = f[d] - c;
    }
    for (int q = 0; q < 21; ++q) as[q] = 0.0;
    rho_s = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = ((dx ? t[0] : 1 - t[0]) * (dy ? t[1] : 1 - t[1])) * (dz ? t[2] : 1 - t[2]);
                int64_t node = ((int64_t)(i[2] + dz) * g.ny + (i[1] + dy)) * g.nx + (i[0] + dx);
                for (int q = 0; q < 21; ++q) as[q] += w * a_node(c21, rho, node, q);
                rho_s += w * (double)rho[node];
            }
}

__device__ __forceinline__ void direction(const Grid3D &g, int dir, double n[3]) {
    int k = dir / g.nth, j = dir % g.nth;
    double th = (j + 0.5) * M_PI / g.nth, ph = 2.0 * M_PI * k / g.nph;
    n[0] = sin(th) * cos(ph);
    n[1] = sin(th) * sin(ph);
    n[2] = cos(th);
}

__global__ void k_source3d(Grid3D g, const float *__restrict__ c21, const float *__restrict__ rho,
                           double xs, double ys, double zs, double *__restrict__ gs64, float *__restrict__ src) {
    int dir = blockIdx.x * blockDim.x + threadIdx.x;
    int ndir = g.nph * g.nth;
    if (dir >= ndir) return;
    double as[21], rho_s;
    source_moduli(g, c21, rho, xs, ys, zs, as, rho_s);
    double n[3];
    direction(g, dir, n);
    SrcVel3T<double> r = source_velocity3d(as, n);
    for (int c = 0; c < 3; ++c) gs64[3 * dir + c] = r.V[c] / r.Vn;
    if (dir == 0) {
        double ez[3] = {0.0, 0.0, 1.0};
        SrcVel3T<double> z = source_velocity3d(as, ez);
        for (int q = 0; q < 21; ++q) src[q] = (float)as[q];
        src[21] = (float)rho_s;
        src[22] = (float)z.v;
    }
}

// ------------------------------- velocities ----------------------------------------------------
// At most 170 registers (three 128-thread blocks per SM, as the FP32 loop alone needs; the rarely
// taken FP64 polish would otherwise raise the allocation for every launch).
__global__ void __launch_bounds__(128, 3) k_velocity3d(Grid3D g, const float *__restrict__ a, const float *__restrict__ dax,
                             const float *__restrict__ day, const float *__restrict__ daz,
                             const float *__restrict__ c21, const float *__restrict__ rho,
                             float *__restrict__ vel, float *rate_out) {
    extern __shared__ float tab[];  // sin th, cos th [nth], sin ph, cos ph [nph]
    float *sth = tab, *cth = tab + g.nth, *sph = tab + 2 * g.nth, *cph = tab + 2 * g.nth + g.nph;
    for (int i = threadIdx.x; i < g.nth; i += blockDim.x) {
        double th = (i + 0.5) * M_PI / g.nth;
        sth[i] = (float)sin(th);
        cth[i] = (float)cos(th);
    }
    for (int i = threadIdx.x; i < g.nph; i += blockDim.x) {
        double ph = 2.0 * M_PI * i / g.nph;
        sph[i] = (float)sin(ph);
        cph[i] = (float)cos(ph);
    }
    __syncthreads();
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float mx = 0.f;
    if (node < g.nodes) {
        float A[21], DX[21], DY[21], DZ[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) {
            A[q] = a[(int64_t)q * g.nodes + node];
            DX[q] = dax[(int64_t)q * g.nodes + node];
            DY[q] = day[(int64_t)q * g.nodes + node];
            DZ[q] = daz[(int64_t)q * g.nodes + node];
        }
        int64_t cells = g.nodes * g.nph * g.nth;
        float ihx = (float)(1.0 / g.hx), ihy = (float)(1.0 / g.hy), ihz = (float)(1.0 / g.hz);
        float idth = (float)(1.0 / g.dth), idph = (float)(1.0 / g.dph);
        for (int k = 0; k < g.nph; ++k)
            for (int j = 0; j < g.nth; ++j) {
                float n[3] = {sth[j] * cph[k], sth[j] * sph[k], cth[j]};
                float gap = 1.f;
                RayVel3T<float> r = ray_velocity3d(A, DX, DY, DZ, n, &gap);
                float nth_[3] = {cth[j] * cph[k], cth[j] * sph[k], -sth[j]};
                float td = r.v * (nth_[0] * r.pd[0] + nth_[1] * r.pd[1] + nth_[2] * r.pd[2]);
                float pd = r.v * (-sph[k] * r.pd[0] + cph[k] * r.pd[1]) / sth[j];
                if (!(gap >= QP_GAP_FP64)) {
                    // near a qP-qS degeneracy: the cell in FP64 from the input stiffness and density
                    double ad[21], dxd[21], dyd[21], dzd[21];
                    for (int q = 0; q < 21; ++q) {
                        ad[q] = a_node(c21, rho, node, q);
                        dxd[q] = DX[q];
                        dyd[q] = DY[q];
                        dzd[q] = DZ[q];
                    }
                    const double th = (j + 0.5) * M_PI / g.nth, ph = 2.0 * M_PI * k / g.nph;
                    const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
                    const double nd[3] = {st * cp, st * sp, ct};
                    RayVel3T<double> rd = ray_velocity3d<double>(ad, dxd, dyd, dzd, nd);
                    const double ntd[3] = {ct * cp, ct * sp, -st};
                    td = (float)(rd.v * (ntd[0] * rd.pd[0] + ntd[1] * rd.pd[1] + ntd[2] * rd.pd[2]));
                    pd = (float)(rd.v * (-sp * rd.pd[0] + cp * rd.pd[1]) / st);
                    r.v = (float)rd.v;
                    for (int i = 0; i < 3; ++i) {
                        r.V[i] = (float)rd.V[i];
                        r.pd[i] = (float)rd.pd[i];
                    }
                }
                int64_t o = (int64_t)(k * g.nth + j) * g.nodes + node;
                float out[9] = {r.V[0], r.V[1], r.V[2], td, pd, r.v, r.pd[0], r.pd[1], r.pd[2]};
#pragma unroll
                for (int c = 0; c < 9; ++c) vel[c * cells + o] = out[c];
                float rate = fabsf(r.V[0]) * ihx + fabsf(r.V[1]) * ihy + fabsf(r.V[2]) * ihz +
                             fabsf(td) * idth + fabsf(pd) * idph;
                mx = fmaxf(mx, rate);
            }
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)rate_out, __float_as_int(mx));
}

// ------------------------------- source manifold and initial labels ----------------------------
__global__ void k_frozen3d(Grid3D g, const double *__restrict__ gs64, double xs, double ys, double zs,
                           double r0, double R, uint8_t *__restrict__ frozen) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y % g.ny, iz = blockIdx.y / g.ny, dir = blockIdx.z;
    if (ix >= g.nx) return;
    double gx = gs64[3 * dir], gy = gs64[3 * dir + 1], gz = gs64[3 * dir + 2];
    double dx = __dadd_rn(__dadd_rn(g.ox, __dmul_rn((double)ix, g.hx)), -xs);
    double dy = __dadd_rn(__dadd_rn(g.oy, __dmul_rn((double)iy, g.hy)), -ys);
    double dz = __dadd_rn(__dadd_rn(g.oz, __dmul_rn((double)iz, g.hz)), -zs);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dz, dz), __dmul_rn(dy, dy)), __dmul_rn(dx, dx));
    double dot = __dadd_rn(__dadd_rn(__dmul_rn(dx, gx), __dmul_rn(dy, gy)), __dmul_rn(dz, gz));
    // approaching by more than 1e-12 |d|: on the closest-approach plane d . g_s is rounding noise
    bool approach = dot < 0.0 && __dmul_rn(dot, dot) > __dmul_rn(1e-24, r2);
    bool f = r2 <= __dmul_rn(r0, r0) || (r2 <= __dmul_rn(R, R) && approach);
    frozen[cidx3(g, dir, iz, iy, ix)] = f ? 1 : 0;
}

// Straight-ray data of the local medium (media clamped to the nearest node for ghosts):
// b = d - (d . g) g, n0 = n, tau = n . d / v; q = 1 on the frozen manifold, 0 on the other interior
// cells, and on the ghosts 1 where the straight ray passed its closest approach within R_Sigma.
__global__ void k_init3d(Grid3D g, double xs, double ys, double zs, double R, const float *__restrict__ vel,
                         const uint8_t *__restrict__ frozen, float *b0, float *b1, float *b2) {
    __shared__ double nd[3];
    int dir = blockIdx.z;
    if (threadIdx.x == 0) direction(g, dir, nd);
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.pitch) return;
    int ix = c - XPAD3, iy = (int)(blockIdx.y % g.rows) - 2, iz = (int)(blockIdx.y / g.rows) - 2;
    int cx = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
    int cy = iy < 0 ? 0 : (iy >= g.ny ? g.ny - 1 : iy);
    int cz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
    int64_t cells = g.nodes * g.nph * g.nth;
    int64_t o = cidx3(g, dir, cz, cy, cx);
    double V[3] = {(double)vel[o], (double)vel[cells + o], (double)vel[2 * cells + o]};
    double v = (double)vel[5 * cells + o];
    double Vn = sqrt(V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
    double gg[3] = {V[0] / Vn, V[1] / Vn, V[2] / Vn};
    double d[3] = {g.ox + ix * g.hx - xs, g.oy + iy * g.hy - ys, g.oz + iz * g.hz - zs};
    double dg = d[0] * gg[0] + d[1] * gg[1] + d[2] * gg[2];
    double tau = (nd[0] * d[0] + nd[1] * d[1] + nd[2] * d[2]) / v;
    bool interior = ix >= 0 && ix < g.nx && iy >= 0 && iy < g.ny && iz >= 0 && iz < g.nz;
    double bv[3] = {d[0] - dg * gg[0], d[1] - dg * gg[1], d[2] - dg * gg[2]};
    float q;
    if (interior) {
        q = frozen[cidx3(g, dir, iz, iy, ix)] ? 1.f : 0.f;
    } else {
        // ghosts continue the source-ray tube: 1 where the straight ray passed its closest approach
        // within R_Sigma (not approaching the source), 0 elsewhere
        double bn = sqrt(bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2]);
        double r2 = d[2] * d[2] + d[1] * d[1] + d[0] * d[0];
        bool approach = dg < 0.0 && dg * dg > 1e-24 * r2;
        q = (bn <= R && !approach) ? 1.f : 0.f;
    }
    float hi = (float)tau;
    float lo = (float)(tau - (double)hi);
    float vals[NF3] = {(float)bv[0], (float)bv[1], (float)bv[2],
                       (float)nd[0], (float)nd[1], (float)nd[2], q, hi, lo};
    int64_t p = (int64_t)dir * g.block + ((int64_t)blockIdx.y) * g.pitch + c;
#pragma unroll
    for (int f = 0; f < NF3; ++f) {
        b0[f * g.field + p] = vals[f];
        b1[f * g.field + p] = vals[f];
        b2[f * g.field + p] = vals[f];
    }
}

cudaError_t solve3d_setup(Solve3D &sv, float *d_rate, cudaStream_t s) {
    const Grid3D &g = sv.g;
    int ndir = g.nph * g.nth;
    const Medium &m = *sv.m;
    k_source3d<<<(ndir + 127) / 128, 128, 0, s>>>(g, m.c21, m.rho, sv.xs[0], sv.xs[1], sv.xs[2], sv.gs64, sv.src);
    size_t tab = (size_t)(2 * g.nth + 2 * g.nph) * sizeof(float);
    k_velocity3d<<<(unsigned)((g.nodes + 127) / 128), 128, tab, s>>>(g, m.a, m.dadx, m.dady, m.dadz, m.c21, m.rho,
                                                                     sv.vel, d_rate);
    dim3 gf((g.nx + 127) / 128, g.ny * g.nz, ndir);
    k_frozen3d<<<gf, 128, 0, s>>>(g, sv.gs64, sv.xs[0], sv.xs[1], sv.xs[2], sv.r0, sv.R_sigma, sv.frozen);
    dim3 gi((g.pitch + 127) / 128, (g.nz + 4) * g.rows, ndir);
    k_init3d<<<gi, 128, 0, s>>>(g, sv.xs[0], sv.xs[1], sv.xs[2], sv.R_sigma, sv.vel, sv.frozen, sv.state[0], sv.state[1],
                                sv.state[2]);
    return cudaGetLastError();
}

// ------------------------------- stencil -------------------------------------------------------
struct Stage3Args {
    Grid3D g;
    const float *in;   // stage input
    const float *un;   // u^n
    float *out;
    const float *vel;  // [9][cells]
    const uint8_t *frozen;
    float dt, coef;
    float ih[5];       // 1/hx, 1/hy, 1/hz, 1/dth, 1/dph
    float eps[4];      // b, n0, q, tau
};

// Work decomposition: blockIdx.x = direction cell (fastest, so that the CTAs resident at a time
// cover many directions of one spatial tile and the theta/phi neighbours of a cell are read from L2),
// blockIdx.y = (2 blockDim.x) x blockDim.y tile in (x, y), blockIdx.z = chunk of ZC3 z slices marched
// by the CTA (the z neighbours of the next slice are the ones just read).  The tile shape is chosen
// per grid (tile_shape3d).
constexpr int ZC3 = 8;
constexpr int MAXT3 = 256;  // threads per block at most (64 registers: 4 such blocks per SM)

template <int STAGE>
__global__ void __launch_bounds__(MAXT3, 4) k_rk3_3d(Stage3Args A) {
    const Grid3D &g = A.g;
    const int px = blockDim.x;  // x pairs per tile row
    int nxt = (g.nx + 2 * px - 1) / (2 * px);
    int dir = blockIdx.x;
    int ix = 2 * ((blockIdx.y % nxt) * px + threadIdx.x);
    int iy = (blockIdx.y / nxt) * blockDim.y + threadIdx.y;
    if (ix >= g.nx || iy >= g.ny) return;
    int zend = min((int)(blockIdx.z + 1) * ZC3, g.nz);
    for (int iz = blockIdx.z * ZC3; iz < zend; ++iz) {
    int k = dir / g.nth, j = dir % g.nth;
    bool second = ix + 1 < g.nx;
    int64_t cells = g.nodes * g.nph * g.nth;
    int64_t o0 = cidx3(g, dir, iz, iy, ix), o1 = second ? o0 + 1 : o0;
    float2 vv[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) vv[c] = f2(A.vel[c * cells + o0], A.vel[c * cells + o1]);
    const bool fa = A.frozen[o0] != 0, fb = A.frozen[o1] != 0;
    const int64_t p = pidx3(g, dir, iz, iy, ix);
    int64_t tn[5], pn[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        tn[m] = (int64_t)theta_neighbour(g, k, j, m - 2) * g.block + (p - (int64_t)dir * g.block);
        pn[m] = (int64_t)phi_neighbour(g, k, j, m - 2) * g.block + (p - (int64_t)dir * g.block);
    }
    const int64_t sy = g.pitch, sz = (int64_t)g.rows * g.pitch;
    auto gather = [&](int f, float2 s[5][5]) {
        const float *F = A.in + (int64_t)f * g.field;
        float2 a = *reinterpret_cast<const float2 *>(F + p - 2);
        float2 b = *reinterpret_cast<const float2 *>(F + p);
        float2 e = *reinterpret_cast<const float2 *>(F + p + 2);
        s[0][0] = a; s[0][1] = f2(a.y, b.x); s[0][2] = b; s[0][3] = f2(b.y, e.x); s[0][4] = e;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            s[1][m] = *reinterpret_cast<const float2 *>(F + p + (m - 2) * sy);
            s[2][m] = *reinterpret_cast<const float2 *>(F + p + (m - 2) * sz);
            s[3][m] = *reinterpret_cast<const float2 *>(F + tn[m]);
            s[4][m] = *reinterpret_cast<const float2 *>(F + pn[m]);
        }
    };
    // upwind sides and -V_d / (2 h_d) per dimension, shared by the nine fields
    Up2 up[5];
    float2 cc[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        up[d] = upwind2(vv[d]);
        const float c = -0.5f * A.ih[d];
        cc[d] = mul2(vv[d], f2(c, c));
    }
    auto rhs_of = [&](const float2 du[5]) {  // -(V . grad u) from the 2 h u_d of weno()
        float2 acc = mul2(cc[0], du[0]);
#pragma unroll
        for (int d = 1; d < 5; ++d) acc = fma2(cc[d], du[d], acc);
        return acc;
    };
    const float2 dt2 = f2(A.dt, A.dt), cf2 = f2(A.coef, A.coef);
#pragma unroll 1
    for (int f = 0; f < 7; ++f) {
        float2 s[5][5];
        gather(f, s);
        float eps = A.eps[f < 3 ? 0 : (f < 6 ? 1 : 2)];
        float2 du[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) du[d] = deriv(s[d], up[d], f2(eps, eps));
        float2 L = rhs_of(du);
        float2 uc = s[0][2];
        float2 un = (STAGE == 1) ? uc : *reinterpret_cast<const float2 *>(A.un + (int64_t)f * g.field + p);
        float2 o = fma2(cf2, fma2(dt2, L, sub2(uc, un)), un);
        float2 r = f2(fa ? un.x : o.x, fb ? un.y : o.y);
        float *O = A.out + (int64_t)f * g.field + p;
        if (second) *reinterpret_cast<float2 *>(O) = r;
        else *O = r.x;
    }
    {
        float2 sh[5][5], sl[5][5];
        gather(7, sh);
        gather(8, sl);
        float2 du[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) du[d] = deriv_ff(sh[d], sl[d], up[d], f2(A.eps[3], A.eps[3]));
        float2 L = add2(rhs_of(du), f2(1.f, 1.f));
        float2 hc = sh[0][2], lc = sl[0][2];
        float2 hn = hc, ln = lc;
        if (STAGE != 1) {
            hn = *reinterpret_cast<const float2 *>(A.un + 7 * g.field + p);
            ln = *reinterpret_cast<const float2 *>(A.un + 8 * g.field + p);
        }
        float2 inc = mul2(cf2, fma2(dt2, L, add2(sub2(hc, hn), sub2(lc, ln))));
        ff ra = ff_add_f(hn.x, ln.x, inc.x);
        ff rb = ff_add_f(hn.y, ln.y, inc.y);
        const float2 r7 = f2(fa ? hn.x : ra.hi, fb ? hn.y : rb.hi);
        const float2 r8 = f2(fa ? ln.x : ra.lo, fb ? ln.y : rb.lo);
        float *O = A.out + 7 * g.field + p;
        if (second) {
            *reinterpret_cast<float2 *>(O) = r7;
            *reinterpret_cast<float2 *>(O + g.field) = r8;
        } else {
            O[0] = r7.x;
            O[g.field] = r8.x;
        }
    }
    }
}

// Thread tile of k_rk3_3d for an nx x ny plane: 128 threads as 32 x pairs by 4 rows, or 16 by 8 when
// that covers nx with fewer idle cells (ties keep the longer rows).  Measured on the two triclinic
// sizes (evolution cell-updates/s, 48^3 x 12 x 24 / 96^3 x 24 x 48): 32 x 4 3.83e9 / 3.22e9,
// 16 x 8 3.68e9 / 3.42e9, 32 x 8 3.68e9 / 3.33e9, 16 x 16 3.54e9 / 3.41e9, 8 x 16 3.40e9 / 2.65e9:
// shorter rows cost more in locality (L2 hits, DRAM re-reads) than idle lanes cost in issue slots.
static dim3 tile_shape3d(int nx, int /*ny*/) {
    const int w32 = 64 * ((nx + 63) / 64), w16 = 32 * ((nx + 31) / 32);
    return w16 < w32 ? dim3(16, 8) : dim3(32, 4);
}

cudaError_t solve3d_evolve(Solve3D &sv, int steps, cudaStream_t s) {
    const Grid3D &g = sv.g;
    Stage3Args A;
    A.g = g;
    A.vel = sv.vel;
    A.frozen = sv.frozen;
    A.dt = (float)sv.dt;
    double ih[5] = {1.0 / g.hx, 1.0 / g.hy, 1.0 / g.hz, 1.0 / g.dth, 1.0 / g.dph};
    for (int d = 0; d < 5; ++d) A.ih[d] = (float)ih[d];
    double h = fmax(g.hx, fmax(g.hy, g.hz));
    A.eps[0] = (float)(1e-6 * h * h);
    A.eps[1] = 1e-6f;
    A.eps[2] = 1e-6f;
    A.eps[3] = (float)(1e-6 * (h / sv.c_ref) * (h / sv.c_ref));
    dim3 block = tile_shape3d(g.nx, g.ny);
    const int tw = 2 * (int)block.x, th = (int)block.y;
    dim3 grid(g.nph * g.nth, ((g.nx + tw - 1) / tw) * ((g.ny + th - 1) / th), (g.nz + ZC3 - 1) / ZC3);
    float *U = sv.state[0], *B = sv.state[1], *C = sv.state[2];
    for (int st = 0; st < steps; ++st) {
        A.un = U;
        A.in = U; A.out = B; A.coef = 1.f;
        k_rk3_3d<1><<<grid, block, 0, s>>>(A);
        A.in = B; A.out = C; A.coef = 0.25f;
        k_rk3_3d<2><<<grid, block, 0, s>>>(A);
        A.in = C; A.out = U; A.coef = (float)(2.0 / 3.0);
        k_rk3_3d<3><<<grid, block, 0, s>>>(A);
    }
    return cudaGetLastError();
}

__global__ void k_read_state3d(Grid3D g, const float *__restrict__ st, double *out) {
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y % g.ny, iz = blockIdx.y / g.ny, dir = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t p = pidx3(g, dir, iz, iy, ix);
    int64_t o = cidx3(g, dir, iz, iy, ix);
    int64_t cells = g.nodes * g.nph * g.nth;
    for (int f = 0; f < 7; ++f) out[f * cells + o] = (double)st[f * g.field + p];
    out[7 * cells + o] = (double)st[7 * g.field + p] + (double)st[8 * g.field + p];
}

cudaError_t launch_read_state3d(const Solve3D &sv, double *out_dev, cudaStream_t s) {
    const Grid3D &g = sv.g;
    dim3 grid((g.nx + 127) / 128, g.ny * g.nz, g.nph * g.nth);
    k_read_state3d<<<grid, 128, 0, s>>>(g, sv.state[0], out_dev);
    return cudaGetLastError();
}

// ------------------------------- superposition -------------------------------------------------
struct Sup3Args {
    Grid3D g;
    const float *st;      // u^n
    const float *vel;     // [9][cells]
    const float *rho;     // [nodes]
    const float *src;     // a_s[21], rho_s, c_ref
    const double *gs64;   // [dir][3]
    const uint8_t *frozen;
    uint8_t *FL;          // [cells] source flag
    int pln;              // max(nx, ny, nz): planes per family in the slot table
    int *cnt;             // [3 pln ndir] centres found per (family, plane, direction)
    int4 *rec;            // [slots][KC3] (triangle id, w0, w1, w2 bits)
    float4 *geo;          // [slots][KC3] in-plane centre position (2), in-plane slowness (2)
    float4 *dat;          // [n_omega][slots][KC3][2]: (E, M11), (M12 + M21, M22)
    int n_omega;
    const double *omega_dev;
    double w0, xs, ys, zs, r0;
    float C1, C2, C3;
    unsigned *err;
};

__global__ void k_flags3d(Sup3Args A) {
    const Grid3D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y % g.ny, iz = blockIdx.y / g.ny, dir = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t o = cidx3(g, dir, iz, iy, ix);
    float q = A.st[6 * g.field + pidx3(g, dir, iz, iy, ix)];
    A.FL[o] = (q > 0.5f && !A.frozen[o]) ? 1 : 0;
}

// Everything the dynamic ray tracing needs at a point of Gamma, interpolated from the vertex cells
// of a triangle (FP64): label gradients with the angular part as an ambient tangent vector.
struct PointData {
    double gb[3][6], gn[3][6];
    double n0[3], V[3], ndot[3], n[3], pdot[3];
    double v, rho, tau;
};

__device__ __forceinline__ float Fat(const Sup3Args &A, int f, int dir, int iz, int iy, int ix) {
    return A.st[(int64_t)f * A.g.field + pidx3(A.g, dir, iz, iy, ix)];
}

// centred difference along a spatial axis, second order one-sided at the grid edges
__device__ __forceinline__ double dspace(const Sup3Args &A, int f, int dir, int iz, int iy, int ix, int axis) {
    const Grid3D &g = A.g;
    int i = axis == 0 ? ix : (axis == 1 ? iy : iz);
    int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    double h = axis == 0 ? g.hx : (axis == 1 ? g.hy : g.hz);
    auto F = [&](int m) {
        return (double)(axis == 0 ? Fat(A, f, dir, iz, iy, m) : (axis == 1 ? Fat(A, f, dir, iz, m, ix) : Fat(A, f, dir, m, iy, ix)));
    };
    if (i == 0) return (4.0 * (F(1) - F(0)) - (F(2) - F(0))) / (2.0 * h);
    if (i == n - 1) return (4.0 * (F(n - 1) - F(n - 2)) - (F(n - 1) - F(n - 3))) / (2.0 * h);
    return (F(i + 1) - F(i - 1)) / (2.0 * h);
}

__device__ void grad6(const Sup3Args &A, int f, int dir, int iz, int iy, int ix, double out[6]) {
    const Grid3D &g = A.g;
    int k = dir / g.nth, j = dir % g.nth;
    out[0] = dspace(A, f, dir, iz, iy, ix, 0);
    out[1] = dspace(A, f, dir, iz, iy, ix, 1);
    out[2] = dspace(A, f, dir, iz, iy, ix, 2);
    double ut = ((double)Fat(A, f, theta_neighbour(g, k, j, 1), iz, iy, ix) -
                 (double)Fat(A, f, theta_neighbour(g, k, j, -1), iz, iy, ix)) / (2.0 * g.dth);
    double up = ((double)Fat(A, f, phi_neighbour(g, k, j, 1), iz, iy, ix) -
                 (double)Fat(A, f, phi_neighbour(g, k, j, -1), iz, iy, ix)) / (2.0 * g.dph);
    double th = (j + 0.5) * M_PI / g.nth, ph = 2.0 * M_PI * k / g.nph;
    double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
    double n_th[3] = {ct * cp, ct * sp, -st}, e_ph[3] = {-sp, cp, 0.0};
    for (int c = 0; c < 3; ++c) out[3 + c] = ut * n_th[c] + up / st * e_ph[c];
}

__device__ void gather_point(const Sup3Args &A, const int cell[3][4], const double w[3], PointData &P) {
    const Grid3D &g = A.g;
    int64_t cells = g.nodes * g.nph * g.nth;
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 6; ++c) { P.gb[a][c] = 0.0; P.gn[a][c] = 0.0; }
        P.n0[a] = P.V[a] = P.ndot[a] = P.n[a] = P.pdot[a] = 0.0;
    }
    P.v = P.rho = P.tau = 0.0;
    for (int vtx = 0; vtx < 3; ++vtx) {
        int dir = cell[vtx][0], iz = cell[vtx][1], iy = cell[vtx][2], ix = cell[vtx][3];
        double wv = w[vtx];
        double gtmp[6];
        for (int a = 0; a < 3; ++a) {
            grad6(A, a, dir, iz, iy, ix, gtmp);
            for (int c = 0; c < 6; ++c) P.gb[a][c] += wv * gtmp[c];
            grad6(A, 3 + a, dir, iz, iy, ix, gtmp);
            for (int c = 0; c < 6; ++c) P.gn[a][c] += wv * gtmp[c];
            P.n0[a] += wv * (double)Fat(A, 3 + a, dir, iz, iy, ix);
        }
        int64_t o = cidx3(g, dir, iz, iy, ix);
        double V[3] = {A.vel[o], A.vel[cells + o], A.vel[2 * cells + o]};
        double td = A.vel[3 * cells + o], pd = A.vel[4 * cells + o];
        int k = dir / g.nth, j = dir % g.nth;
        double th = (j + 0.5) * M_PI / g.nth, ph = 2.0 * M_PI * k / g.nph;
        double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
        double n[3] = {st * cp, st * sp, ct}, n_th[3] = {ct * cp, ct * sp, -st}, e_ph[3] = {-sp, cp, 0.0};
        for (int c = 0; c < 3; ++c) {
            P.V[c] += wv * V[c];
            P.n[c] += wv * n[c];
            P.ndot[c] += wv * (td * n_th[c] + pd * st * e_ph[c]);
            P.pdot[c] += wv * (double)A.vel[(6 + c) * cells + o];
        }
        P.v += wv * (double)A.vel[5 * cells + o];
        P.rho += wv * (double)A.rho[((int64_t)iz * g.ny + iy) * g.nx + ix];
        P.tau += wv * ((double)Fat(A, 7, dir, iz, iy, ix) + (double)Fat(A, 8, dir, iz, iy, ix));
    }
}

// Inverse of a 5x5 real matrix by Gauss-Jordan elimination with partial pivoting after row
// equilibration; false if singular.
__device__ bool inv5(double M[5][5], double Inv[5][5]) {
    double a[5][10];
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
        for (int c = 0; c < 5; ++c) s = fmax(s, fabs(M[r][c]));
        if (!(s > 0.0)) return false;
        for (int c = 0; c < 5; ++c) { a[r][c] = M[r][c] / s; a[r][5 + c] = (r == c) ? 1.0 / s : 0.0; }
    }
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (!(fabs(a[piv][c]) > 0.0)) return false;
        if (piv != c)
            for (int q = 0; q < 10; ++q) { double t = a[c][q]; a[c][q] = a[piv][q]; a[piv][q] = t; }
        double d = 1.0 / a[c][c];
        for (int q = 0; q < 10; ++q) a[c][q] *= d;
        for (int r = 0; r < 5; ++r) {
            if (r == c) continue;
            double fct = a[r][c];
            if (fct != 0.0)
                for (int q = 0; q < 10; ++q) a[r][q] -= fct * a[c][q];
        }
    }
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) Inv[r][c] = a[r][5 + c];
    return true;
}

__device__ double det4(double m[4][4]) {
    double a[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) a[r][c] = m[r][c];
    double det = 1.0;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return 0.0;
        if (piv != c) {
            for (int q = 0; q < 4; ++q) { double t = a[c][q]; a[c][q] = a[piv][q]; a[piv][q] = t; }
            det = -det;
        }
        det *= a[c][c];
        for (int r = c + 1; r < 4; ++r) {
            double fct = a[r][c] / a[c][c];
            for (int q = c; q < 4; ++q) a[r][q] -= fct * a[c][q];
        }
    }
    return det;
}

struct Drt {
    double R[5][5], Rinv[5][5];
    double n0[3], vs, Vs[3], Vsn, e1[3], e2[3], f1[3], f2[3], t1[3], t2[3];
    bool ok;
};

// rows R = [e1 . grad b; e2 . grad b; f1 . grad n0; f2 . grad n0; (V, dn/dt)] in (dx, a1, a2)
__device__ void drt_rows(const Sup3Args &A, const double *as, const PointData &P, const double nc[3], Drt &D) {
    double nn = sqrt(P.n0[0] * P.n0[0] + P.n0[1] * P.n0[1] + P.n0[2] * P.n0[2]);
    for (int c = 0; c < 3; ++c) D.n0[c] = P.n0[c] / nn;
    SrcVel3T<double> sv = source_velocity3d(as, D.n0);
    D.vs = sv.v;
    D.Vsn = sv.Vn;
    double G0[3];
    for (int c = 0; c < 3; ++c) { D.Vs[c] = sv.V[c]; G0[c] = sv.V[c] / sv.Vn; }
    frame(G0, D.e1, D.e2);
    frame(D.n0, D.f1, D.f2);
    frame(nc, D.t1, D.t2);
    auto row = [&](const double G[6], double out[5]) {
        out[0] = G[0]; out[1] = G[1]; out[2] = G[2];
        out[3] = G[3] * D.t1[0] + G[4] * D.t1[1] + G[5] * D.t1[2];
        out[4] = G[3] * D.t2[0] + G[4] * D.t2[1] + G[5] * D.t2[2];
    };
    const double *E[2] = {D.e1, D.e2}, *Fv[2] = {D.f1, D.f2};
    for (int r = 0; r < 2; ++r) {
        double Gb[6], Gn[6];
        for (int c = 0; c < 6; ++c) {
            Gb[c] = E[r][0] * P.gb[0][c] + E[r][1] * P.gb[1][c] + E[r][2] * P.gb[2][c];
            Gn[c] = Fv[r][0] * P.gn[0][c] + Fv[r][1] * P.gn[1][c] + Fv[r][2] * P.gn[2][c];
        }
        row(Gb, D.R[r]);
        row(Gn, D.R[2 + r]);
    }
    double Ge[6] = {P.V[0], P.V[1], P.V[2], P.ndot[0], P.ndot[1], P.ndot[2]};
    row(Ge, D.R[4]);
    D.ok = inv5(D.R, D.Rinv);
}

__device__ __forceinline__ double det3(const double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

// ---- arrivals ----
constexpr int KMAX3 = 32;

__global__ void __launch_bounds__(64) k_arrivals3d(Sup3Args A, uint8_t *count, double *T, float *Aout, int kmax) {
    const Grid3D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y, iz = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t node = ((int64_t)iz * g.ny + iy) * g.nx + ix;
    double dn[3] = {g.ox + ix * g.hx - A.xs, g.oy + iy * g.hy - A.ys, g.oz + iz * g.hz - A.zs};
    double r = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
    double Tl[KMAX3];
    float Al[KMAX3];
    int angl[KMAX3];
    int n = 0, total = 0;
    if (r > A.r0) {
        float rh[3] = {(float)(dn[0] / r), (float)(dn[1] / r), (float)(dn[2] / r)};
        float e1[3], e2[3];
        frame(rh, e1, e2);
        double as[21];
        for (int q = 0; q < 21; ++q) as[q] = (double)A.src[q];
        double rho_s = A.src[21], c_ref = A.src[22];
        float rlim = 0.25f * (float)r;
        int ntri_q = 2 * (g.nth - 1) * g.nph;
        int ntri = ntri_q + 2 * (g.nph - 2);
        for (int t = 0; t < ntri; ++t) {
            int vk[3], vj[3];
            if (t < ntri_q) {
                int q = t >> 1, jj = q / g.nph, kk = q % g.nph, k1 = (kk + 1) % g.nph;
                if ((t & 1) == 0) { vk[0] = kk; vj[0] = jj; vk[1] = k1; vj[1] = jj; vk[2] = k1; vj[2] = jj + 1; }
                else { vk[0] = kk; vj[0] = jj; vk[1] = k1; vj[1] = jj + 1; vk[2] = kk; vj[2] = jj + 1; }
            } else {
                int q = t - ntri_q, kk = 1 + (q >> 1);
                if ((q & 1) == 0) { vk[0] = 0; vj[0] = 0; vk[1] = kk + 1; vj[1] = 0; vk[2] = kk; vj[2] = 0; }
                else { int s = g.nth - 1; vk[0] = 0; vj[0] = s; vk[1] = kk; vj[1] = s; vk[2] = kk + 1; vj[2] = s; }
            }
            float P[3][2], br[3];
            bool flagged = true;
            int dirs[3];
            for (int v = 0; v < 3 && flagged; ++v) {
                dirs[v] = vk[v] * g.nth + vj[v];
                int64_t o = cidx3(g, dirs[v], iz, iy, ix);
                if (!A.FL[o]) { flagged = false; break; }
                int64_t p = pidx3(g, dirs[v], iz, iy, ix);
                float b[3] = {A.st[p], A.st[g.field + p], A.st[2 * g.field + p]};
                P[v][0] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
                P[v][1] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
                br[v] = b[0] * rh[0] + b[1] * rh[1] + b[2] * rh[2];
            }
            if (!flagged) continue;
            float w[3];
            if (!origin_in(P, w)) continue;
            float bdot = w[0] * br[0] + w[1] * br[1] + w[2] * br[2];
            if (!(fabsf(bdot) <= rlim)) continue;
            ++total;
            // point-source family of the dynamic ray tracing at the arrival
            int cell[3][4];
            double wd[3] = {w[0], w[1], w[2]};
            for (int v = 0; v < 3; ++v) { cell[v][0] = dirs[v]; cell[v][1] = iz; cell[v][2] = iy; cell[v][3] = ix; }
            PointData Pd;
            gather_point(A, cell, wd, Pd);
            double nc[3];
            double nn = sqrt(Pd.n[0] * Pd.n[0] + Pd.n[1] * Pd.n[1] + Pd.n[2] * Pd.n[2]);
            for (int c = 0; c < 3; ++c) nc[c] = Pd.n[c] / nn;
            Drt D;
            drt_rows(A, as, Pd, nc, D);
            double Xm[3][3];
            for (int c = 0; c < 3; ++c) { Xm[c][0] = D.Rinv[c][2]; Xm[c][1] = D.Rinv[c][3]; Xm[c][2] = Pd.V[c]; }
            double Jps = det3(Xm);
            double Av = c_ref * c_ref * sqrt(rho_s / Pd.rho) / (4.0 * M_PI * pow(D.vs, 1.5) * sqrt(fabs(Jps)));
            if (!D.ok) Av = 0.0;
            int ang = dirs[0];
            double Tv = Pd.tau;
            int pos = n;
            while (pos > 0 && (Tl[pos - 1] > Tv || (Tl[pos - 1] == Tv && angl[pos - 1] > ang))) --pos;
            if (pos < kmax) {
                int last = n < kmax ? n : kmax - 1;
                for (int q = last; q > pos; --q) { Tl[q] = Tl[q - 1]; Al[q] = Al[q - 1]; angl[q] = angl[q - 1]; }
                Tl[pos] = Tv;
                Al[pos] = (float)Av;
                angl[pos] = ang;
                if (n < kmax) ++n;
            }
        }
    }
    if (total > kmax) atomicOr(A.err, DeviceErrors::OVERFLOW);
    if (count) count[node] = (uint8_t)n;
    for (int q = 0; q < kmax; ++q) {
        if (T) T[node * kmax + q] = q < n ? Tl[q] : 0.0;
        if (Aout) Aout[node * kmax + q] = q < n ? Al[q] : 0.f;
    }
}

// ---- beam centres ----
// family 0: planes of constant z (in-plane node indices (iy, ix)); 1: constant y ((iz, ix));
// 2: constant x ((iz, iy)).  Triangles of a quad (i1, i2): ((i1,i2), (i1,i2+1), (i1+1,i2+1)) and
// ((i1,i2), (i1+1,i2+1), (i1+1,i2)).
__device__ __forceinline__ void plane_dims(const Grid3D &g, int fam, int &np, int &n1, int &n2) {
    if (fam == 0) { np = g.nz; n1 = g.ny; n2 = g.nx; }
    else if (fam == 1) { np = g.ny; n1 = g.nz; n2 = g.nx; }
    else { np = g.nx; n1 = g.nz; n2 = g.ny; }
}
__device__ __forceinline__ void plane_node(int fam, int plane, int i1, int i2, int &iz, int &iy, int &ix) {
    if (fam == 0) { iz = plane; iy = i1; ix = i2; }
    else if (fam == 1) { iy = plane; iz = i1; ix = i2; }
    else { ix = plane; iz = i1; iy = i2; }
}
__device__ __forceinline__ void tri_vertices(int t, int i1, int i2, int v1[3], int v2[3]) {
    if (t == 0) { v1[0] = i1; v2[0] = i2; v1[1] = i1; v2[1] = i2 + 1; v1[2] = i1 + 1; v2[2] = i2 + 1; }
    else { v1[0] = i1; v2[0] = i2; v1[1] = i1 + 1; v2[1] = i2 + 1; v1[2] = i1 + 1; v2[2] = i2; }
}

__global__ void k_centres3d(Sup3Args A) {
    const Grid3D &g = A.g;
    int fam = blockIdx.y / A.pln, plane = blockIdx.y % A.pln, dir = blockIdx.z;
    int np, n1, n2;
    plane_dims(g, fam, np, n1, n2);
    if (plane >= np) return;
    int quad = blockIdx.x * blockDim.x + threadIdx.x;
    if (quad >= (n1 - 1) * (n2 - 1)) return;
    int i1 = quad / (n2 - 1), i2 = quad % (n2 - 1);
    float gs[3] = {(float)A.gs64[3 * dir], (float)A.gs64[3 * dir + 1], (float)A.gs64[3 * dir + 2]};
    float e1[3], e2[3];
    frame(gs, e1, e2);
    for (int t = 0; t < 2; ++t) {
        int v1[3], v2[3];
        tri_vertices(t, i1, i2, v1, v2);
        float P[3][2], bg[3], pos[3][3];
        bool flagged = true;
        for (int v = 0; v < 3; ++v) {
            int iz, iy, ix;
            plane_node(fam, plane, v1[v], v2[v], iz, iy, ix);
            if (!A.FL[cidx3(g, dir, iz, iy, ix)]) { flagged = false; break; }
            int64_t p = pidx3(g, dir, iz, iy, ix);
            float b[3] = {A.st[p], A.st[g.field + p], A.st[2 * g.field + p]};
            P[v][0] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
            P[v][1] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
            bg[v] = b[0] * gs[0] + b[1] * gs[1] + b[2] * gs[2];
            pos[v][0] = (float)(g.ox + ix * g.hx - A.xs);
            pos[v][1] = (float)(g.oy + iy * g.hy - A.ys);
            pos[v][2] = (float)(g.oz + iz * g.hz - A.zs);
        }
        if (!flagged) continue;
        float w[3];
        if (!origin_in(P, w)) continue;
        float xc[3];
        for (int c = 0; c < 3; ++c) xc[c] = w[0] * pos[0][c] + w[1] * pos[1][c] + w[2] * pos[2][c];
        float bgc = w[0] * bg[0] + w[1] * bg[1] + w[2] * bg[2];
        if (!(fabsf(bgc) <= 0.25f * sqrtf(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]))) continue;
        int64_t slot = ((int64_t)fam * A.pln + plane) * (g.nph * g.nth) + dir;
        int idx = atomicAdd(&A.cnt[slot], 1);
        if (idx >= KC3) { atomicOr(A.err, DeviceErrors::OVERFLOW); continue; }
        A.rec[slot * KC3 + idx] = make_int4(quad * 2 + t, __float_as_int(w[0]), __float_as_int(w[1]), __float_as_int(w[2]));
    }
}

struct cd { double re, im; };
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd cmuld(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ cd cdivd(cd a, cd b) {
    double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cd csqrtd(cd z) {  // principal branch
    double r = hypot(z.re, z.im);
    double re = sqrt(fmax(0.5 * (r + z.re), 0.0));
    double im = copysign(sqrt(fmax(0.5 * (r - z.re), 0.0)), z.im);
    return {re, im};
}

// omega * tau mod 2 pi with tau = hi + lo, omega = ohi + olo (double-float), Cody-Waite reduction.
__device__ __forceinline__ float phase_mod3(float ohi, float olo, float thi, float tlo, float C1, float C2, float C3) {
    float p = ohi * thi;
    float e = fmaf(ohi, thi, -p);
    e = fmaf(ohi, tlo, e);
    e = fmaf(olo, thi, e);
    float k = rintf(p * 0.159154943091895335769f);
    float r = fmaf(-k, C1, p);
    r = fmaf(-k, C2, r);
    r = fmaf(-k, C3, r);
    return r + e;
}

__global__ void __launch_bounds__(64) k_beam3d(Sup3Args A, int nslots) {
    const Grid3D &g = A.g;
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    int nc = A.cnt[slot];
    nc = nc > KC3 ? KC3 : nc;
    A.cnt[slot] = nc;
    if (nc == 0) return;
    int ndir = g.nph * g.nth;
    int dir = slot % ndir, fp = slot / ndir, plane = fp % A.pln, fam = fp / A.pln;
    int np, n1, n2;
    plane_dims(g, fam, np, n1, n2);
    // deterministic order: by triangle id
    int4 r[KC3];
    for (int i = 0; i < nc; ++i) r[i] = A.rec[(int64_t)slot * KC3 + i];
    for (int i = 1; i < nc; ++i)
        for (int q = i; q > 0 && r[q - 1].x > r[q].x; --q) { int4 t = r[q]; r[q] = r[q - 1]; r[q - 1] = t; }
    int k = dir / g.nth, j = dir % g.nth;
    double th = (j + 0.5) * M_PI / g.nth, ph = 2.0 * M_PI * k / g.nph;
    double n[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
    int c1 = fam == 2 ? 1 : 0, c2 = fam == 0 ? 1 : 2, drop = 2 - fam;
    double as[21];
    for (int q = 0; q < 21; ++q) as[q] = (double)A.src[q];
    double rho_s = A.src[21], c_ref = A.src[22];
    double dOmega = g.dth * g.dph * sin(th);
    for (int i = 0; i < nc; ++i) {
        int quad = r[i].x >> 1, t = r[i].x & 1;
        int i1 = quad / (n2 - 1), i2 = quad % (n2 - 1);
        int v1[3], v2[3];
        tri_vertices(t, i1, i2, v1, v2);
        int cell[3][4];
        double pos[3][3];
        for (int v = 0; v < 3; ++v) {
            int iz, iy, ix;
            plane_node(fam, plane, v1[v], v2[v], iz, iy, ix);
            cell[v][0] = dir; cell[v][1] = iz; cell[v][2] = iy; cell[v][3] = ix;
            pos[v][0] = g.ox + ix * g.hx - A.xs;
            pos[v][1] = g.oy + iy * g.hy - A.ys;
            pos[v][2] = g.oz + iz * g.hz - A.zs;
        }
        double w[3] = {__int_as_float(r[i].y), __int_as_float(r[i].z), __int_as_float(r[i].w)};
        double xc[3];
        for (int c = 0; c < 3; ++c) xc[c] = w[0] * pos[0][c] + w[1] * pos[1][c] + w[2] * pos[2][c];
        PointData P;
        gather_point(A, cell, w, P);
        Drt D;
        drt_rows(A, as, P, n, D);
        double v = P.v;
        double p[3] = {n[0] / v, n[1] / v, n[2] / v};
        double dpa[2][3];
        const double *tt[2] = {D.t1, D.t2};
        for (int a = 0; a < 2; ++a) {
            double Vt = P.V[0] * tt[a][0] + P.V[1] * tt[a][1] + P.V[2] * tt[a][2];
            for (int c = 0; c < 3; ++c) dpa[a][c] = tt[a][c] / v - n[c] * Vt / (v * v);
        }
        // pairing of offsets with take-off rotations (source Hessian i c Pi^T Pi)
        const double *E[2] = {D.e1, D.e2}, *F[2] = {D.f1, D.f2};
        double Am[2][2], Pe[2][3], Q[2][2];
        double n0e[2], Vsf[2];
        for (int a = 0; a < 2; ++a) Vsf[a] = D.Vs[0] * F[a][0] + D.Vs[1] * F[a][1] + D.Vs[2] * F[a][2];
        for (int a = 0; a < 2; ++a) {
            n0e[a] = D.n0[0] * E[a][0] + D.n0[1] * E[a][1] + D.n0[2] * E[a][2];
            for (int b = 0; b < 2; ++b)
                Am[a][b] = (E[a][0] * F[b][0] + E[a][1] * F[b][1] + E[a][2] * F[b][2]) / D.vs - n0e[a] * Vsf[b] / (D.vs * D.vs);
            for (int c = 0; c < 3; ++c) Pe[a][c] = E[a][c] - D.Vs[c] * n0e[a] / D.vs;
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) Q[a][b] = Pe[a][0] * Pe[b][0] + Pe[a][1] * Pe[b][1] + Pe[a][2] * Pe[b][2];
        double detA = Am[0][0] * Am[1][1] - Am[0][1] * Am[1][0];
        double AQ[2][2];
        for (int b = 0; b < 2; ++b) {
            AQ[0][b] = (Am[1][1] * Q[0][b] - Am[0][1] * Q[1][b]) / detA;
            AQ[1][b] = (-Am[1][0] * Q[0][b] + Am[0][0] * Q[1][b]) / detA;
        }
        // plane blend times the take-off measure
        double dets[3];
        for (int a = 0; a < 3; ++a) {
            int ca = a == 0 ? 1 : 0, cb = a == 2 ? 1 : 2;
            dets[a] = D.R[0][ca] * D.R[1][cb] - D.R[0][cb] * D.R[1][ca];
        }
        double Ssum = dets[0] * dets[0] + dets[1] * dets[1] + dets[2] * dets[2];
        double Ja[4][4];
        int cols[4] = {c1, c2, 3, 4};
        for (int rr = 0; rr < 4; ++rr)
            for (int cc = 0; cc < 4; ++cc) Ja[rr][cc] = D.R[rr][cols[cc]];
        double wj = fabs(dets[drop]) * fabs(det4(Ja)) / Ssum;
        int64_t ci = (int64_t)slot * KC3 + i;
        A.geo[ci] = make_float4((float)xc[c1], (float)xc[c2], (float)p[c1], (float)p[c2]);
        int64_t cstride = (int64_t)nslots * KC3;
        for (int wi = 0; wi < A.n_omega; ++wi) {
            double om = A.omega_dev[wi];
            double cc = 2.0 / (om * A.w0 * A.w0);
            cd dx[2][3], dpj[2][3];
            for (int jj = 0; jj < 2; ++jj) {
                cd d5[5];
                for (int q = 0; q < 5; ++q)
                    d5[q] = {D.Rinv[q][jj], cc * (AQ[0][jj] * D.Rinv[q][2] + AQ[1][jj] * D.Rinv[q][3])};
                cd pdx = {0.0, 0.0};
                for (int c = 0; c < 3; ++c) { dx[jj][c] = d5[c]; pdx = cadd(pdx, cscale(d5[c], P.pdot[c])); }
                for (int c = 0; c < 3; ++c)
                    dpj[jj][c] = cadd(cadd(cscale(pdx, p[c]), cscale(d5[3], dpa[0][c])), cscale(d5[4], dpa[1][c]));
            }
            // X = [dx1 dx2 V], Pm = [dp1 dp2 pdot]; J = det X; M = Pm X^-1
            cd X[3][3], Pm[3][3];
            for (int c = 0; c < 3; ++c) {
                X[c][0] = dx[0][c]; X[c][1] = dx[1][c]; X[c][2] = {P.V[c], 0.0};
                Pm[c][0] = dpj[0][c]; Pm[c][1] = dpj[1][c]; Pm[c][2] = {P.pdot[c], 0.0};
            }
            auto m2 = [&](int a, int b, int c, int d) { return csub(cmuld(X[a][b], X[c][d]), cmuld(X[a][d], X[c][b])); };
            cd adj[3][3];  // adjugate: adj[i][j] = cofactor(j, i)
            adj[0][0] = m2(1, 1, 2, 2); adj[0][1] = cscale(m2(0, 1, 2, 2), -1.0); adj[0][2] = m2(0, 1, 1, 2);
            adj[1][0] = cscale(m2(1, 0, 2, 2), -1.0); adj[1][1] = m2(0, 0, 2, 2); adj[1][2] = cscale(m2(0, 0, 1, 2), -1.0);
            adj[2][0] = m2(1, 0, 2, 1); adj[2][1] = cscale(m2(0, 0, 2, 1), -1.0); adj[2][2] = m2(0, 0, 1, 1);
            cd J = cadd(cadd(cmuld(X[0][0], adj[0][0]), cmuld(X[0][1], adj[1][0])), cmuld(X[0][2], adj[2][0]));
            auto Mel = [&](int a, int b) {
                cd s = {0.0, 0.0};
                for (int q = 0; q < 3; ++q) s = cadd(s, cmuld(Pm[a][q], adj[q][b]));
                return cdivd(s, J);
            };
            cd M11 = Mel(c1, c1), Mx = cadd(Mel(c1, c2), Mel(c2, c1)), M22 = Mel(c2, c2);
            double sigma = atan2(J.im, J.re) < -1e-3 ? -1.0 : 1.0;
            cd amp = cscale(csqrtd(cdivd(cd{rho_s * D.Vsn / P.rho, 0.0}, J)), sigma);
            double wreal = om * c_ref * c_ref * dOmega * wj / (8.0 * M_PI * M_PI * D.vs * D.vs * D.vs);
            cd coef = {-wreal * amp.im, wreal * amp.re};
            float ohi = (float)om, olo = (float)(om - (double)ohi);
            float thi = (float)P.tau, tlo = (float)(P.tau - (double)thi);
            float phs = phase_mod3(ohi, olo, thi, tlo, A.C1, A.C2, A.C3);
            float sp, cp;
            sincosf(phs, &sp, &cp);
            cd Ec = cmuld(coef, cd{cp, sp});
            bool fin = D.ok && isfinite(Ec.re) && isfinite(Ec.im) && isfinite(M11.re) && isfinite(M11.im) &&
                       isfinite(Mx.re) && isfinite(Mx.im) && isfinite(M22.re) && isfinite(M22.im);
            float4 d0 = fin ? make_float4((float)Ec.re, (float)Ec.im, (float)M11.re, (float)M11.im) : make_float4(0, 0, 0, 0);
            float4 d1 = fin ? make_float4((float)Mx.re, (float)Mx.im, (float)M22.re, (float)M22.im) : make_float4(0, 0, 0, 0);
            A.dat[2 * ((int64_t)wi * cstride + ci)] = d0;
            A.dat[2 * ((int64_t)wi * cstride + ci) + 1] = d1;
        }
    }
}

__global__ void k_sum3d(Sup3Args A, float2 *u, int nslots) {
    const Grid3D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y, iz = blockIdx.z;
    if (ix >= g.nx) return;
    int ndir = g.nph * g.nth;
    float xr[3] = {(float)(g.ox + ix * g.hx - A.xs), (float)(g.oy + iy * g.hy - A.ys), (float)(g.oz + iz * g.hz - A.zs)};
    int64_t cstride = (int64_t)nslots * KC3;
    for (int wi = 0; wi < A.n_omega; ++wi) {
        float om = (float)A.omega_dev[wi];
        float are = 0.f, aim = 0.f;
        for (int fam = 0; fam < 3; ++fam) {
            int plane = fam == 0 ? iz : (fam == 1 ? iy : ix);
            int c1 = fam == 2 ? 1 : 0, c2 = fam == 0 ? 1 : 2;
            int64_t base = ((int64_t)fam * A.pln + plane) * ndir;
            for (int dir = 0; dir < ndir; ++dir) {
                int64_t slot = base + dir;
                int nc = A.cnt[slot];
                for (int i = 0; i < nc; ++i) {
                    int64_t ci = slot * KC3 + i;
                    float4 geo = A.geo[ci];
                    float4 d0 = A.dat[2 * ((int64_t)wi * cstride + ci)];
                    float4 d1 = A.dat[2 * ((int64_t)wi * cstride + ci) + 1];
                    float a1 = xr[c1] - geo.x, a2 = xr[c2] - geo.y;
                    float qre = d0.z * a1 * a1 + d1.x * a1 * a2 + d1.z * a2 * a2;
                    float qim = d0.w * a1 * a1 + d1.y * a1 * a2 + d1.w * a2 * a2;
                    float dec = -0.5f * om * fmaxf(qim, 0.f);
                    if (dec < -60.f) continue;
                    float ph = om * (geo.z * a1 + geo.w * a2 + 0.5f * qre);
                    float mag = __expf(dec);
                    float sp, cp;
                    sincosf(ph, &sp, &cp);
                    are += mag * (d0.x * cp - d0.y * sp);
                    aim += mag * (d0.x * sp + d0.y * cp);
                }
            }
        }
        u[((int64_t)wi * g.nz + iz) * g.ny * g.nx + (int64_t)iy * g.nx + ix] = make_float2(are, aim);
    }
}

static int planes_max(const Grid3D &g) {
    int m = g.nx > g.ny ? g.nx : g.ny;
    return m > g.nz ? m : g.nz;
}

size_t superpose3d_scratch_bytes(const Solve3D &sv) {
    const Grid3D &g = sv.g;
    size_t cells = (size_t)g.nodes * g.nph * g.nth;
    size_t slots = (size_t)3 * planes_max(g) * g.nph * g.nth;
    size_t no = sv.omega.size();
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(cells) + al(slots * 4) + al(slots * KC3 * 16) + al(slots * KC3 * 16) +
           al(no * slots * KC3 * 32) + al(no * 8) + 4096;
}

static void split_two_pi3(float &C1, float &C2, float &C3) {
    const double two_pi = 6.283185307179586476925286766559;
    auto trunc_bits = [](double x, int bits) {
        int e;
        double m = frexp(x, &e);
        double sc = ldexp(1.0, bits);
        return ldexp(floor(m * sc) / sc, e);
    };
    double c1 = trunc_bits(two_pi, 15);
    double c2 = trunc_bits(two_pi - c1, 15);
    C1 = (float)c1;
    C2 = (float)c2;
    C3 = (float)(two_pi - c1 - c2);
}

cudaError_t launch_superpose3d(Solve3D &sv, float2 *u_dev, uint8_t *count_dev, double *T_dev, float *A_dev,
                               int kmax, unsigned *d_err, cudaStream_t s) {
    const Grid3D &g = sv.g;
    size_t cells = (size_t)g.nodes * g.nph * g.nth;
    int pln = planes_max(g);
    int ndir = g.nph * g.nth;
    size_t slots = (size_t)3 * pln * ndir;
    size_t no = sv.omega.size();
    char *base = (char *)sv.scratch;
    auto take = [&](size_t bytes) {
        char *p = base;
        base += (bytes + 255) & ~(size_t)255;
        return (void *)p;
    };
    Sup3Args A;
    A.g = g;
    A.st = sv.state[0];
    A.vel = sv.vel;
    A.rho = sv.m->rho;
    A.src = sv.src;
    A.gs64 = sv.gs64;
    A.frozen = sv.frozen;
    A.FL = (uint8_t *)take(cells);
    A.pln = pln;
    A.cnt = (int *)take(slots * 4);
    A.rec = (int4 *)take(slots * KC3 * 16);
    A.geo = (float4 *)take(slots * KC3 * 16);
    A.dat = (float4 *)take(no * slots * KC3 * 32);
    double *om = (double *)take(no * 8);
    if ((size_t)(base - (char *)sv.scratch) > sv.scratch_bytes) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(om, sv.omega.data(), no * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    A.n_omega = (int)no;
    A.omega_dev = om;
    A.w0 = sv.w0;
    A.xs = sv.xs[0];
    A.ys = sv.xs[1];
    A.zs = sv.xs[2];
    A.r0 = sv.r0;
    split_two_pi3(A.C1, A.C2, A.C3);
    A.err = d_err;
    k_flags3d<<<dim3((g.nx + 127) / 128, g.ny * g.nz, ndir), 128, 0, s>>>(A);
    if (u_dev) {
        e = cudaMemsetAsync(A.cnt, 0, slots * 4, s);
        if (e != cudaSuccess) return e;
        int maxq = 0;
        for (int fam = 0; fam < 3; ++fam) {
            int n1 = fam == 0 ? g.ny : g.nz, n2 = fam == 2 ? g.ny : g.nx;
            int q = (n1 - 1) * (n2 - 1);
            maxq = q > maxq ? q : maxq;
        }
        k_centres3d<<<dim3((maxq + 127) / 128, 3 * pln, ndir), 128, 0, s>>>(A);
        k_beam3d<<<(unsigned)((slots + 63) / 64), 64, 0, s>>>(A, (int)slots);
        k_sum3d<<<dim3((g.nx + 63) / 64, g.ny, g.nz), 64, 0, s>>>(A, u_dev, (int)slots);
    }
    if (count_dev || T_dev || A_dev)
        k_arrivals3d<<<dim3((g.nx + 63) / 64, g.ny, g.nz), 64, 0, s>>>(A, count_dev, T_dev, A_dev, kmax);
    return cudaGetLastError();
}

}  // namespace egb
