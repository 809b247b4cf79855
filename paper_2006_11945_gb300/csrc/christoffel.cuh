// qP Christoffel eigenpair and ray velocities in FP32 (device code).
//
// Eq. 4: Gamma_ik = a_ijkl n_j n_l; Eq. 3: the qP phase velocity is v = sqrt(lambda_max(Gamma(n))),
// g the unit eigenvector (polarisation); Eq. 7: p = n / v with n = (sin theta, 0, cos theta).
// Ray velocities of H = (lambda(Gamma(x, p)) - 1) / 2 (traveltime parametrisation):
//   V_i = a_ijkl p_l g_j g_k,   dp_i/dt = -1/2 g . Gamma(d_i a, p) . g,
//   dtheta/dt = v (cos theta dp_x/dt - sin theta dp_z/dt).
// The largest eigenvalue comes from the trigonometric solution of the characteristic cubic
// (Smith, CACM 4(4) 1961), the eigenvector from the largest cross product of two rows of
// Gamma - lambda I, and one Rayleigh-quotient pass refines both.
#pragma once

#include "egb_internal.cuh"

namespace egb {

struct Sym3 { float xx, yy, zz, xy, xz, yz; };

// Gamma(n) for n = (s, 0, c): Gamma_ik = a_i0k0 s^2 + (a_i0k2 + a_i2k0) s c + a_i2k2 c^2.
__device__ __forceinline__ float gam(const float *a, int i, int k, float s, float c) {
    return a[aidx(i, 0, k, 0)] * s * s + (a[aidx(i, 0, k, 2)] + a[aidx(i, 2, k, 0)]) * s * c +
           a[aidx(i, 2, k, 2)] * c * c;
}

__device__ __forceinline__ Sym3 christoffel2d(const float *a, float s, float c) {
    Sym3 G;
    G.xx = gam(a, 0, 0, s, c);
    G.yy = gam(a, 1, 1, s, c);
    G.zz = gam(a, 2, 2, s, c);
    G.xy = gam(a, 0, 1, s, c);
    G.xz = gam(a, 0, 2, s, c);
    G.yz = gam(a, 1, 2, s, c);
    return G;
}

__device__ __forceinline__ float quad(const Sym3 &G, const float g[3]) {
    return G.xx * g[0] * g[0] + G.yy * g[1] * g[1] + G.zz * g[2] * g[2] +
           2.f * (G.xy * g[0] * g[1] + G.xz * g[0] * g[2] + G.yz * g[1] * g[2]);
}

__device__ __forceinline__ void eigvec_for(const Sym3 &G, float lam, float g[3]) {
    float r0[3] = {G.xx - lam, G.xy, G.xz};
    float r1[3] = {G.xy, G.yy - lam, G.yz};
    float r2[3] = {G.xz, G.yz, G.zz - lam};
    float c01[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]};
    float c02[3] = {r0[1] * r2[2] - r0[2] * r2[1], r0[2] * r2[0] - r0[0] * r2[2], r0[0] * r2[1] - r0[1] * r2[0]};
    float c12[3] = {r1[1] * r2[2] - r1[2] * r2[1], r1[2] * r2[0] - r1[0] * r2[2], r1[0] * r2[1] - r1[1] * r2[0]};
    float n01 = c01[0] * c01[0] + c01[1] * c01[1] + c01[2] * c01[2];
    float n02 = c02[0] * c02[0] + c02[1] * c02[1] + c02[2] * c02[2];
    float n12 = c12[0] * c12[0] + c12[1] * c12[1] + c12[2] * c12[2];
    const float *best = c01;
    float nb = n01;
    if (n02 > nb) { best = c02; nb = n02; }
    if (n12 > nb) { best = c12; nb = n12; }
    float inv = rsqrtf(fmaxf(nb, 1e-37f));
    g[0] = best[0] * inv;
    g[1] = best[1] * inv;
    g[2] = best[2] * inv;
}

// Largest eigenvalue and unit eigenvector of a symmetric 3x3 matrix (qP branch).
__device__ __forceinline__ float qp_eigen(const Sym3 &G, float g[3]) {
    float m = (G.xx + G.yy + G.zz) * (1.f / 3.f);
    float b00 = G.xx - m, b11 = G.yy - m, b22 = G.zz - m;
    float p2 = (b00 * b00 + b11 * b11 + b22 * b22 +
                2.f * (G.xy * G.xy + G.xz * G.xz + G.yz * G.yz)) * (1.f / 6.f);
    float lam;
    if (p2 <= 0.f) {
        lam = m;
    } else {
        float p = sqrtf(p2);
        float det = b00 * (b11 * b22 - G.yz * G.yz) - G.xy * (G.xy * b22 - G.yz * G.xz) +
                    G.xz * (G.xy * G.yz - b11 * G.xz);
        float r = det / (2.f * p2 * p);
        r = fminf(1.f, fmaxf(-1.f, r));
        float phi = acosf(r) * (1.f / 3.f);
        lam = m + 2.f * p * cosf(phi);
    }
    eigvec_for(G, lam, g);
    lam = quad(G, g);
    eigvec_for(G, lam, g);
    return quad(G, g);
}

// V_i = (1/v) sum_jk g_j g_k (a_ijk0 s + a_ijk2 c) for i = 0 (x) or 2 (z).
template <int I>
__device__ __forceinline__ float group_component(const float *a, const float g[3], float s, float c) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            acc += g[j] * g[k] * (a[aidx(I, j, k, 0)] * s + a[aidx(I, j, k, 2)] * c);
    return acc;
}

struct RayVel { float v, Vx, Vz, pdx, pdz, td; };

// Full per-cell solve: phase velocity, group velocity, dp/dt, dtheta/dt.
__device__ __forceinline__ RayVel ray_velocity2d(const float *a, const float *dax, const float *daz,
                                                 float s, float c) {
    Sym3 G = christoffel2d(a, s, c);
    float g[3];
    float lam = qp_eigen(G, g);
    RayVel r;
    r.v = sqrtf(lam);
    float iv = 1.f / r.v;
    r.Vx = group_component<0>(a, g, s, c) * iv;
    r.Vz = group_component<2>(a, g, s, c) * iv;
    float iv2 = iv * iv;
    r.pdx = -0.5f * quad(christoffel2d(dax, s, c), g) * iv2;
    r.pdz = -0.5f * quad(christoffel2d(daz, s, c), g) * iv2;
    r.td = r.v * (c * r.pdx - s * r.pdz);
    return r;
}

struct SrcVel { float v, Vx, Vz, Vn; };

// Source-medium quantities at phase angle theta (no gradients).
__device__ __forceinline__ SrcVel source_velocity(const float *a, float s, float c) {
    Sym3 G = christoffel2d(a, s, c);
    float g[3];
    float lam = qp_eigen(G, g);
    SrcVel r;
    r.v = sqrtf(lam);
    float iv = 1.f / r.v;
    r.Vx = group_component<0>(a, g, s, c) * iv;
    r.Vz = group_component<2>(a, g, s, c) * iv;
    r.Vn = sqrtf(r.Vx * r.Vx + r.Vz * r.Vz);
    return r;
}

}  // namespace egb
