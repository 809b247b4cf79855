// qP Christoffel eigenpair and ray velocities (device code; R = float for the production path,
// R = double for the plain all-FP64 form).
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

template <typename R> struct Sym3T { R xx, yy, zz, xy, xz, yz; };
using Sym3 = Sym3T<float>;

// Gamma(n) for n = (s, 0, c): Gamma_ik = a_i0k0 s^2 + (a_i0k2 + a_i2k0) s c + a_i2k2 c^2.
template <typename R>
__device__ __forceinline__ R gam(const R *a, int i, int k, R s, R c) {
    return a[aidx(i, 0, k, 0)] * s * s + (a[aidx(i, 0, k, 2)] + a[aidx(i, 2, k, 0)]) * s * c +
           a[aidx(i, 2, k, 2)] * c * c;
}

template <typename R>
__device__ __forceinline__ Sym3T<R> christoffel2d(const R *a, R s, R c) {
    Sym3T<R> G;
    G.xx = gam(a, 0, 0, s, c);
    G.yy = gam(a, 1, 1, s, c);
    G.zz = gam(a, 2, 2, s, c);
    G.xy = gam(a, 0, 1, s, c);
    G.xz = gam(a, 0, 2, s, c);
    G.yz = gam(a, 1, 2, s, c);
    return G;
}

template <typename R>
__device__ __forceinline__ R quad(const Sym3T<R> &G, const R g[3]) {
    return G.xx * g[0] * g[0] + G.yy * g[1] * g[1] + G.zz * g[2] * g[2] +
           R(2) * (G.xy * g[0] * g[1] + G.xz * g[0] * g[2] + G.yz * g[1] * g[2]);
}

template <typename R>
__device__ __forceinline__ void eigvec_for(const Sym3T<R> &G, R lam, R g[3]) {
    R r0[3] = {G.xx - lam, G.xy, G.xz};
    R r1[3] = {G.xy, G.yy - lam, G.yz};
    R r2[3] = {G.xz, G.yz, G.zz - lam};
    R c01[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]};
    R c02[3] = {r0[1] * r2[2] - r0[2] * r2[1], r0[2] * r2[0] - r0[0] * r2[2], r0[0] * r2[1] - r0[1] * r2[0]};
    R c12[3] = {r1[1] * r2[2] - r1[2] * r2[1], r1[2] * r2[0] - r1[0] * r2[2], r1[0] * r2[1] - r1[1] * r2[0]};
    R n01 = c01[0] * c01[0] + c01[1] * c01[1] + c01[2] * c01[2];
    R n02 = c02[0] * c02[0] + c02[1] * c02[1] + c02[2] * c02[2];
    R n12 = c12[0] * c12[0] + c12[1] * c12[1] + c12[2] * c12[2];
    const R *best = c01;
    R nb = n01;
    if (n02 > nb) { best = c02; nb = n02; }
    if (n12 > nb) { best = c12; nb = n12; }
    R inv = R(1) / sqrt(nb > R(1e-37) ? nb : R(1e-37));
    g[0] = best[0] * inv;
    g[1] = best[1] * inv;
    g[2] = best[2] * inv;
}

// Relative gap (lambda_1 - lambda_2) / lambda_1 between the two largest eigenvalues below which the
// FP32 path recomputes a cell in FP64 from the input moduli: near a qP-qS degeneracy the eigenvector
// is sensitive to rounding as (rounding) / gap, and at a gap of 1e-5 FP32 moduli and arithmetic
// cost about 5e-5 in the group velocity (1.5e-7 at gaps of 2e-3 and more).
constexpr float QP_GAP_FP64 = 1e-3f;

// Largest eigenvalue and unit eigenvector of a symmetric 3x3 matrix (qP branch); with rel_gap, also
// the relative gap to the second eigenvalue from the same trigonometric roots (0 when all three
// coincide).
template <typename R>
__device__ __forceinline__ R qp_eigen(const Sym3T<R> &G, R g[3], R *rel_gap = nullptr) {
    R m = (G.xx + G.yy + G.zz) * (R(1) / R(3));
    R b00 = G.xx - m, b11 = G.yy - m, b22 = G.zz - m;
    R p2 = (b00 * b00 + b11 * b11 + b22 * b22 +
            R(2) * (G.xy * G.xy + G.xz * G.xz + G.yz * G.yz)) * (R(1) / R(6));
    R lam;
    if (p2 <= R(0)) {
        lam = m;
        if (rel_gap) *rel_gap = R(0);
    } else {
        R p = sqrt(p2);
        R det = b00 * (b11 * b22 - G.yz * G.yz) - G.xy * (G.xy * b22 - G.yz * G.xz) +
                G.xz * (G.xy * G.yz - b11 * G.xz);
        R r = det / (R(2) * p2 * p);
        r = r > R(1) ? R(1) : (r < R(-1) ? R(-1) : r);
        R phi = acos(r) * (R(1) / R(3));
        const R cphi = cos(phi);
        lam = m + R(2) * p * cphi;
        if (rel_gap) {
            // lambda_1 - lambda_2 = 2 sqrt(3) p sin(pi/3 - phi) = 3 p cos phi - sqrt(3) p sin phi,
            // with phi in [0, pi/3] so that sin phi = sqrt(1 - cos^2 phi)
            const R s2 = R(1) - cphi * cphi;
            const R sphi = sqrt(s2 > R(0) ? s2 : R(0));
            *rel_gap = (R(3) * cphi - R(1.7320508075688772935) * sphi) * p / lam;
        }
    }
    eigvec_for(G, lam, g);
    lam = quad(G, g);
    eigvec_for(G, lam, g);
    return quad(G, g);
}

// V_i = (1/v) sum_jk g_j g_k (a_ijk0 s + a_ijk2 c) for i = 0 (x) or 2 (z).
template <int I, typename R>
__device__ __forceinline__ R group_component(const R *a, const R g[3], R s, R c) {
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            acc += g[j] * g[k] * (a[aidx(I, j, k, 0)] * s + a[aidx(I, j, k, 2)] * c);
    return acc;
}

template <typename R> struct RayVelT { R v, Vx, Vz, pdx, pdz, td; };
using RayVel = RayVelT<float>;

// Full per-cell solve: phase velocity, group velocity, dp/dt, dtheta/dt.
template <typename R>
__device__ __forceinline__ RayVelT<R> ray_velocity2d(const R *a, const R *dax, const R *daz, R s, R c,
                                                     R *rel_gap = nullptr) {
    Sym3T<R> G = christoffel2d(a, s, c);
    R g[3];
    R lam = qp_eigen(G, g, rel_gap);
    RayVelT<R> r;
    r.v = sqrt(lam);
    R iv = R(1) / r.v;
    r.Vx = group_component<0>(a, g, s, c) * iv;
    r.Vz = group_component<2>(a, g, s, c) * iv;
    R iv2 = iv * iv;
    r.pdx = R(-0.5) * quad(christoffel2d(dax, s, c), g) * iv2;
    r.pdz = R(-0.5) * quad(christoffel2d(daz, s, c), g) * iv2;
    r.td = r.v * (c * r.pdx - s * r.pdz);
    return r;
}

template <typename R> struct SrcVelT { R v, Vx, Vz, Vn; };
using SrcVel = SrcVelT<float>;

// Source-medium quantities at phase angle theta (no gradients).
template <typename R>
__device__ __forceinline__ SrcVelT<R> source_velocity(const R *a, R s, R c, R *rel_gap = nullptr) {
    Sym3T<R> G = christoffel2d(a, s, c);
    R g[3];
    R lam = qp_eigen(G, g, rel_gap);
    SrcVelT<R> r;
    r.v = sqrt(lam);
    R iv = R(1) / r.v;
    r.Vx = group_component<0>(a, g, s, c) * iv;
    r.Vz = group_component<2>(a, g, s, c) * iv;
    r.Vn = sqrt(r.Vx * r.Vx + r.Vz * r.Vz);
    return r;
}

// ---- general 3-D direction n ----------------------------------------------------------------
// Gamma_ik = sum_jl a_ijkl n_j n_l
template <typename R>
__device__ __forceinline__ R gam3(const R *a, int i, int k, const R n[3]) {
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int l = 0; l < 3; ++l) acc += a[aidx(i, j, k, l)] * n[j] * n[l];
    return acc;
}

template <typename R>
__device__ __forceinline__ Sym3T<R> christoffel3d(const R *a, const R n[3]) {
    Sym3T<R> G;
    G.xx = gam3(a, 0, 0, n);
    G.yy = gam3(a, 1, 1, n);
    G.zz = gam3(a, 2, 2, n);
    G.xy = gam3(a, 0, 1, n);
    G.xz = gam3(a, 0, 2, n);
    G.yz = gam3(a, 1, 2, n);
    return G;
}

// sum_jk g_j g_k sum_l a_ijkl n_l (= v V_i on the unit direction n)
template <typename R>
__device__ __forceinline__ R group3(const R *a, const R g[3], const R n[3], int i) {
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R t = R(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) t += a[aidx(i, j, k, l)] * n[l];
            acc += g[j] * g[k] * t;
        }
    return acc;
}

template <typename R> struct RayVel3T { R v, V[3], pd[3]; };

// Phase velocity, group velocity and dp/dt at the unit direction n: V_i = a_ijkl p_l g_j g_k,
// dp_i/dt = -1/2 g . Gamma(d_i a, p) . g with p = n / v.
template <typename R>
__device__ __forceinline__ RayVel3T<R> ray_velocity3d(const R *a, const R *dax, const R *day, const R *daz,
                                                      const R n[3], R *rel_gap = nullptr) {
    Sym3T<R> G = christoffel3d(a, n);
    R g[3];
    R lam = qp_eigen(G, g, rel_gap);
    RayVel3T<R> r;
    r.v = sqrt(lam);
    R iv = R(1) / r.v, iv2 = iv * iv;
#pragma unroll
    for (int i = 0; i < 3; ++i) r.V[i] = group3(a, g, n, i) * iv;
    r.pd[0] = R(-0.5) * quad(christoffel3d(dax, n), g) * iv2;
    r.pd[1] = R(-0.5) * quad(christoffel3d(day, n), g) * iv2;
    r.pd[2] = R(-0.5) * quad(christoffel3d(daz, n), g) * iv2;
    return r;
}

template <typename R> struct SrcVel3T { R v, V[3], Vn; };

template <typename R>
__device__ __forceinline__ SrcVel3T<R> source_velocity3d(const R *a, const R n[3]) {
    Sym3T<R> G = christoffel3d(a, n);
    R g[3];
    R lam = qp_eigen(G, g);
    SrcVel3T<R> r;
    r.v = sqrt(lam);
    R iv = R(1) / r.v;
#pragma unroll
    for (int i = 0; i < 3; ++i) r.V[i] = group3(a, g, n, i) * iv;
    r.Vn = sqrt(r.V[0] * r.V[0] + r.V[1] * r.V[1] + r.V[2] * r.V[2]);
    return r;
}

}  // namespace egb
