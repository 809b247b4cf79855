// Paraxial depth march of the level sets (Sec. 3-4, Eqs. 13-20) and its same-row Gaussian-beam
// superposition (Sec. 5, Eqs. 25-28, 33-35), two-sided from the source row: the paper's own
// formulation, for rays that keep their vertical direction.
//
// Each branch s (+1 down, -1 up) marches zeta = s (z - z_s) over the (theta, x) plane of one depth:
//   phi_zeta + U phi_x + W phi_theta = S_phi,  U = s Vx/Vz, W = s thetadot/Vz (Eqs. 14-15, 17-18),
//   S_tau = s/Vz (Eq. 19's p_3 + p_1 dx/dz = p.V/Vz), S = 0 for the labels,
// from D = x - x_s (the position label X of Eq. 20 relative to the source), vartheta = theta,
// tau = 0 on the source row; phase angles theta_k = -theta_max + (k + 1/2) dtheta (+ pi upward).
//
//  k_zm_coef      per node of the branch's rows, every angle: qP group velocity and phase-angle rate
//                 (Eqs. 8-12) -> U, W, S and the superposition's Vx, Vz, v, dp_x/dt; the largest CFL
//                 rate; a latched error where s Vz <= 0 (Eq. 13 violated)
//  k_zm_init      Eq. 20 on the source row (also its history row), source indicator q = 1
//  k_zm_stage<S>  one Shu-Osher stage of one depth substep: third-order HJ-WENO in x and theta,
//                 differences beyond the ends clamped to the outermost one (identical to ghost cells
//                 holding the linear extrapolation of the two outermost values), coefficients
//                 interpolated linearly between the two rows; the source indicator q is advected
//                 with ghost cells holding 0 (rays entering through a boundary carry no source-plane
//                 data); the last stage of a row records the row's labels in the history volume
//  k_zm_centres   per (row, angle): sign changes of D along x between cells with q > 1/2 are
//                 beam centres; dynamic ray tracing
//                 from the label gradients at fixed depth (the perturbation with db = 1 and the
//                 initial transverse beam Hessian of Eq. 24) -> M_xx (Eq. 25), spreading and amplitude
//                 (Eq. 26), weight (Eq. 33), exp(i omega tau) reduced in double-float
//  k_zm_sum       per receiver: sum over the beams centred on its row (Eq. 34)
//  k_zm_arrivals  per receiver: sign changes of D along theta (q > 1/2) -> traveltime and amplitude
//                 of every arrival (late arrivals included)
#include <algorithm>
#include <cmath>
#include <cstring>

#include "christoffel.cuh"

namespace egb {

namespace zm {

struct Geom {
    int nx, nth, nr, js, s;  // grid, angles, rows of the branch, source row, branch sign
    double hx, hz, ox, xs;
    float dth;
};

// rows r of a branch sit at depth index js + s r
__device__ __forceinline__ int row_index(const Geom &G, int r) { return G.js + G.s * r; }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Third-order HJ-WENO (Jiang-Peng) from the four differences d_0..d_3 of a five-point stencil, in
// second-difference form: e_j = d_{j+1} - d_j, e_up = e_0 (flow towards +) or e_2, A = e_up^2 + eps,
// B = e_1^2 + eps, w = B^2 / (B^2 + 2 A^2); returns 2 h u_x = d_1 + d_2 +/- w (e_up - e_1).
__device__ __forceinline__ float weno2h(const float d[4], bool left, float eps) {
    float e0 = d[1] - d[0], e1 = d[2] - d[1], e2 = d[3] - d[2];
    float E = left ? e0 : e2;
    float A = fmaf(E, E, eps), B = fmaf(e1, e1, eps);
    float B2 = B * B;
    float w = __fdividef(B2, fmaf(2.f * A, A, B2));
    return fmaf(left ? w : -w, E - e1, d[1] + d[2]);
}

struct StageArgs {
    Geom G;
    float ihx, idth, h, t, coef;
    float eps[4];               // D, vartheta, tau, q
    const float *c0, *c1;       // coefficient rows r and r + 1 (U plane; W, S at +cst, +2 cst)
    int64_t cst;                // floats between the U, W and S planes of the table
    const float *in, *un;       // [5][nth][nx]: D, vartheta, tau_hi, tau_lo, q
    float *out;
    float *hist;                // history row to record (D plane of row r + 1), or null
    int64_t hfield, hk;         // history strides: per field, per angle
    // advected dynamic ray tracing (Eq. 21): Jacobian rows r, r + 1 of (U, W) in (x, theta)
    // (U_x plane; U_theta, W_x, W_theta at +cst, +2 cst, +3 cst); Q fields are planes 5..8 of the
    // state and history (dx_1, dtheta_1, dx_2, dtheta_2)
    const float *j0, *j1;
    float qeps[4];
};

constexpr int NF_LABELS = 5;   // D, vartheta, tau_hi, tau_lo, q
constexpr int NF_DRT = 9;      // + dx_1, dtheta_1, dx_2, dtheta_2

template <int STAGE, bool QDRT>
__device__ __forceinline__ void stage_body(const StageArgs &A, int k, int i) {
    const int nx = A.G.nx, nth = A.G.nth;
    const int64_t P = (int64_t)nth * nx;
    const int64_t c = (int64_t)k * nx + i;
    const float U = fmaf(A.t, A.c1[c] - A.c0[c], A.c0[c]);
    const float W = fmaf(A.t, A.c1[A.cst + c] - A.c0[A.cst + c], A.c0[A.cst + c]);
    const float S = fmaf(A.t, A.c1[2 * A.cst + c] - A.c0[2 * A.cst + c], A.c0[2 * A.cst + c]);
    const bool lx = U > 0.f, lt = W > 0.f;
    // -U / (2 hx), -W / (2 dtheta) turn weno2h's 2 h u_x into -U u_x, -W u_theta
    const float cx = -0.5f * U * A.ihx, ct = -0.5f * W * A.idth;
    int ix[4], it[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ix[j] = clampi(i + j - 2, 0, nx - 2);
        it[j] = clampi(k + j - 2, 0, nth - 2);
    }
    float L[3];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const float *F = A.in + f * P;
        float dx[4], dt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            dx[j] = F[(int64_t)k * nx + ix[j] + 1] - F[(int64_t)k * nx + ix[j]];
            dt[j] = F[(int64_t)(it[j] + 1) * nx + i] - F[(int64_t)it[j] * nx + i];
        }
        L[f] = fmaf(cx, weno2h(dx, lx, A.eps[f]), ct * weno2h(dt, lt, A.eps[f]));
    }
    {
        const float *Hh = A.in + 2 * P, *Hl = A.in + 3 * P;
        float dx[4], dt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t a0 = (int64_t)k * nx + ix[j], b0 = (int64_t)it[j] * nx + i;
            dx[j] = (Hh[a0 + 1] - Hh[a0]) + (Hl[a0 + 1] - Hl[a0]);
            dt[j] = (Hh[b0 + nx] - Hh[b0]) + (Hl[b0 + nx] - Hl[b0]);
        }
        L[2] = S + fmaf(cx, weno2h(dx, lx, A.eps[2]), ct * weno2h(dt, lt, A.eps[2]));
    }
    float Lq;
    {
        // source indicator: its ghost cells hold 0 (rays entering through a boundary)
        const float *F = A.in + 4 * P;
        auto qv = [&](int kk, int ii) {
            return (kk < 0 || kk >= nth || ii < 0 || ii >= nx) ? 0.f : F[(int64_t)kk * nx + ii];
        };
        float sx[5], st[5], dx[4], dt[4];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            sx[j] = qv(k, i + j - 2);
            st[j] = qv(k + j - 2, i);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            dx[j] = sx[j + 1] - sx[j];
            dt[j] = st[j + 1] - st[j];
        }
        Lq = fmaf(cx, weno2h(dx, lx, A.eps[3]), ct * weno2h(dt, lt, A.eps[3]));
    }
    float o[5];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        float u = A.in[f * P + c];
        float n = (STAGE == 1) ? u : A.un[f * P + c];
        o[f] = fmaf(A.coef, fmaf(A.h, L[f], u - n), n);
    }
    {
        float hi = A.in[2 * P + c], lo = A.in[3 * P + c];
        float hn = (STAGE == 1) ? hi : A.un[2 * P + c], ln = (STAGE == 1) ? lo : A.un[3 * P + c];
        float inc = A.coef * fmaf(A.h, L[2], (hi - hn) + (lo - ln));
        ff r = ff_add_f(hn, ln, inc);
        o[2] = r.hi;
        o[3] = r.lo;
    }
    {
        float u = A.in[4 * P + c];
        float n = (STAGE == 1) ? u : A.un[4 * P + c];
        o[4] = fmaf(A.coef, fmaf(A.h, Lq, u - n), n);
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) A.out[f * P + c] = o[f];
    if (STAGE == 3 && A.hist) {
#pragma unroll
        for (int f = 0; f < 5; ++f) A.hist[f * A.hfield + (int64_t)k * A.hk + i] = o[f];
    }
    if (QDRT) {
        // Q_zeta + U Q_x + W Q_theta = J Q for the two perturbation families (Eq. 21 in the march's
        // variables), ghosts by linear extrapolation (clamped differences) like the labels
        float J[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            J[e] = fmaf(A.t, A.j1[e * A.cst + c] - A.j0[e * A.cst + c], A.j0[e * A.cst + c]);
        float Lq4[4], qv[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float *F = A.in + (5 + f) * P;
            float dx[4], dt[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                dx[j] = F[(int64_t)k * nx + ix[j] + 1] - F[(int64_t)k * nx + ix[j]];
                dt[j] = F[(int64_t)(it[j] + 1) * nx + i] - F[(int64_t)it[j] * nx + i];
            }
            Lq4[f] = fmaf(cx, weno2h(dx, lx, A.qeps[f]), ct * weno2h(dt, lt, A.qeps[f]));
            qv[f] = F[c];
        }
#pragma unroll
        for (int fam = 0; fam < 2; ++fam) {
            const float qx = qv[2 * fam], qt = qv[2 * fam + 1];
            Lq4[2 * fam] += fmaf(J[0], qx, J[1] * qt);
            Lq4[2 * fam + 1] += fmaf(J[2], qx, J[3] * qt);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            float u = qv[f];
            float n = (STAGE == 1) ? u : A.un[(5 + f) * P + c];
            float ov = fmaf(A.coef, fmaf(A.h, Lq4[f], u - n), n);
            A.out[(5 + f) * P + c] = ov;
            if (STAGE == 3 && A.hist) A.hist[(5 + f) * A.hfield + (int64_t)k * A.hk + i] = ov;
        }
    }
}

// One stage over the (theta, x) planes of one or two branches (blockIdx.z selects the branch): the
// two branches are independent until the superposition, so advancing both in one launch doubles the
// cells a launch covers.  Stages are launched as programmatic dependents of the one before: every
// CTA first lets the next stage's grid begin launching (it can start only once all CTAs of this one
// are running, so it never takes their slots), then waits until the previous grid has completed and
// its writes are visible, before any load or store.
template <int STAGE, bool QDRT>
__global__ void __launch_bounds__(128) k_zm_stage(const __grid_constant__ StageArgs A0,
                                                  const __grid_constant__ StageArgs A1) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const StageArgs &A = blockIdx.z ? A1 : A0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (i < A.G.nx && k < A.G.nth) stage_body<STAGE, QDRT>(A, k, i);
}

// Jacobian of the characteristic field (U, W) in (x, theta) on every cell of the branch's rows:
// second-order centred differences of the tabulated U, W, one-sided at the ends (as for the labels).
// Jt: [4][nr][nth][nx] (U_x, U_theta, W_x, W_theta).
__global__ void k_zm_jac(Geom G, const float *C, float *Jt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y, k = blockIdx.z;
    if (i >= G.nx) return;
    const int64_t T = (int64_t)G.nr * G.nth * G.nx;
    const int nx = G.nx, nth = G.nth;
    const float ihx = (float)(0.5 / G.hx), idt = 0.5f / G.dth;
    auto at = [&](int comp, int kk, int ii) { return C[comp * T + ((int64_t)r * nth + kk) * nx + ii]; };
    auto gx = [&](int comp) {
        if (i == 0) return (4.f * (at(comp, k, 1) - at(comp, k, 0)) - (at(comp, k, 2) - at(comp, k, 0))) * ihx;
        if (i == nx - 1) return (4.f * (at(comp, k, nx - 1) - at(comp, k, nx - 2)) - (at(comp, k, nx - 1) - at(comp, k, nx - 3))) * ihx;
        return (at(comp, k, i + 1) - at(comp, k, i - 1)) * ihx;
    };
    auto gt = [&](int comp) {
        if (k == 0) return (4.f * (at(comp, 1, i) - at(comp, 0, i)) - (at(comp, 2, i) - at(comp, 0, i))) * idt;
        if (k == nth - 1) return (4.f * (at(comp, nth - 1, i) - at(comp, nth - 2, i)) - (at(comp, nth - 1, i) - at(comp, nth - 3, i))) * idt;
        return (at(comp, k + 1, i) - at(comp, k - 1, i)) * idt;
    };
    const int64_t o = ((int64_t)r * nth + k) * nx + i;
    Jt[o] = gx(0);
    Jt[T + o] = gt(0);
    Jt[2 * T + o] = gx(1);
    Jt[3 * T + o] = gt(1);
}

__global__ void k_zm_init(Geom G, const float2 *sc, const double *theta, const float *src, int nf,
                          float *st, float *hist, int64_t hfield, int64_t hk) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (i >= G.nx) return;
    int64_t P = (int64_t)G.nth * G.nx, c = (int64_t)k * G.nx + i;
    float v[NF_DRT] = {(float)(G.ox + i * G.hx - G.xs), (float)theta[k], 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    if (nf > NF_LABELS) {
        // offset family Q1 = (1 / ghat_z, 0) of the source medium at theta_k; Q2 = (0, 1)
        float as[21];
        for (int q = 0; q < 21; ++q) as[q] = src[q];
        SrcVel sv = source_velocity(as, sc[k].x, sc[k].y);
        v[5] = sv.Vn / sv.Vz;
    }
    for (int f = 0; f < nf; ++f) {
        st[f * P + c] = v[f];
        hist[f * hfield + (int64_t)k * hk + i] = v[f];
    }
}

// Coefficient and velocity tables of a branch: one thread per node of its rows, every angle.
// C: [3][nr][nth][nx] (U, W, S); V: [4][nr][nth][nx] (Vx, Vz, v, dp_x/dt).
__global__ void k_zm_coef(Medium m, Geom G, const float2 *sc, float *C, float *V, float *rate,
                          unsigned *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    float rmax = 0.f;
    if (i < G.nx) {
        int nodes = m.nx * m.nz;
        int node = row_index(G, r) * m.nx + i;
        float a[21], dx[21], dz[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) {
            a[q] = m.a[(int64_t)q * nodes + node];
            dx[q] = m.dadx[(int64_t)q * nodes + node];
            dz[q] = m.dadz[(int64_t)q * nodes + node];
        }
        int64_t T = (int64_t)G.nr * G.nth * G.nx;
        float ihx = (float)(1.0 / G.hx), idth = 1.f / G.dth, sg = (float)G.s;
        bool bad = false;
        for (int k = 0; k < G.nth; ++k) {
            RayVel rv = ray_velocity2d(a, dx, dz, sc[k].x, sc[k].y);
            int64_t o = ((int64_t)r * G.nth + k) * G.nx + i;
            float U = 0.f, W = 0.f, S = 0.f;
            if (sg * rv.Vz > 0.f) {
                float iv = sg / rv.Vz;
                U = rv.Vx * iv;
                W = rv.td * iv;
                S = iv;
            } else {
                bad = true;
            }
            C[o] = U;
            C[T + o] = W;
            C[2 * T + o] = S;
            V[o] = rv.Vx;
            V[T + o] = rv.Vz;
            V[2 * T + o] = rv.v;
            V[3 * T + o] = rv.pdx;
            rmax = fmaxf(rmax, fabsf(U) * ihx + fabsf(W) * idth);
        }
        if (bad) atomicOr(err, DeviceErrors::PARAXIAL);
    }
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    __shared__ float wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wmax[w]);
        atomicMax((int *)rate, __float_as_int(b));
    }
}

// ---- superposition on the history volume H[4][nth][nr][nx] ----
struct SupArgsZ {
    Geom G;
    const float *H;             // history
    int64_t hf;                 // floats per history field
    const float *V;             // [4][nr][nth][nx]
    int64_t vt;                 // floats per velocity plane
    const float *rho;           // medium density [nz][nx]
    const float *src;           // source block: a_s, rho_s, c_ref
    const float2 *sc;           // sin, cos of theta_k
    int *cnt;                   // [nr][nth] beam centres per line
    float *pos, *px;            // [nr][nth][KC]
    float4 *dat;                // [n_omega][nr][nth][KC]: E.re, E.im, M.re, max(M.im, 0)
    int n_omega;
    const double *omega;
    float w0;
    float C1, C2, C3;
    unsigned *err;
    int drt;                    // 1: perturbations from the advected Q fields (history planes 5..8)
};

__device__ __forceinline__ float hval(const SupArgsZ &A, int f, int k, int r, int i) {
    return A.H[f * A.hf + ((int64_t)k * A.G.nr + r) * A.G.nx + i];
}

// second-order centred difference, second-order one-sided at the two ends (n >= 3)
__device__ __forceinline__ float grad_x(const SupArgsZ &A, int f, int k, int r, int i, float ih) {
    int n = A.G.nx;
    if (i == 0) return (4.f * (hval(A, f, k, r, 1) - hval(A, f, k, r, 0)) - (hval(A, f, k, r, 2) - hval(A, f, k, r, 0))) * 0.5f * ih;
    if (i == n - 1) return (4.f * (hval(A, f, k, r, n - 1) - hval(A, f, k, r, n - 2)) - (hval(A, f, k, r, n - 1) - hval(A, f, k, r, n - 3))) * 0.5f * ih;
    return (hval(A, f, k, r, i + 1) - hval(A, f, k, r, i - 1)) * 0.5f * ih;
}
__device__ __forceinline__ float grad_t(const SupArgsZ &A, int f, int k, int r, int i, float ih) {
    int n = A.G.nth;
    if (k == 0) return (4.f * (hval(A, f, 1, r, i) - hval(A, f, 0, r, i)) - (hval(A, f, 2, r, i) - hval(A, f, 0, r, i))) * 0.5f * ih;
    if (k == n - 1) return (4.f * (hval(A, f, n - 1, r, i) - hval(A, f, n - 2, r, i)) - (hval(A, f, n - 1, r, i) - hval(A, f, n - 3, r, i))) * 0.5f * ih;
    return (hval(A, f, k + 1, r, i) - hval(A, f, k - 1, r, i)) * 0.5f * ih;
}

struct cfz { float re, im; };
__device__ __forceinline__ cfz zmul(cfz a, cfz b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cfz zdiv(cfz a, cfz b) {
    float d = 1.f / (b.re * b.re + b.im * b.im);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
__device__ __forceinline__ cfz zsqrt(cfz z) {  // principal branch
    float r = hypotf(z.re, z.im);
    return {sqrtf(fmaxf(0.5f * (r + z.re), 0.f)), copysignf(sqrtf(fmaxf(0.5f * (r - z.re), 0.f)), z.im)};
}
// omega tau mod 2 pi with tau = thi + tlo, omega = ohi + olo (double-float), split-constant reduction
__device__ __forceinline__ float zphase(float ohi, float olo, float thi, float tlo, float C1, float C2,
                                        float C3) {
    float p = ohi * thi;
    float e = fmaf(ohi, thi, -p);
    e = fmaf(ohi, tlo, e);
    e = fmaf(olo, thi, e);
    float q = rintf(p * 0.159154943091895335769f);
    float rr = fmaf(-q, C1, p);
    rr = fmaf(-q, C2, rr);
    rr = fmaf(-q, C3, rr);
    return rr + e;
}

// One line (row r, angle k) per thread.
__global__ void k_zm_centres(SupArgsZ A) {
    const Geom &G = A.G;
    __shared__ float as[21];
    if (threadIdx.x < 21) as[threadIdx.x] = A.src[threadIdx.x];
    __syncthreads();
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= G.nr * G.nth) return;
    int r = line / G.nth, k = line % G.nth;
    const int64_t slot0 = (int64_t)line * KC, total = (int64_t)G.nr * G.nth * KC;
    const float rho_s = A.src[21], c_ref = A.src[22];
    const float ihx = (float)(1.0 / G.hx), idth = 1.f / G.dth, hx = (float)G.hx;
    const float sth = A.sc[k].x, cth = A.sc[k].y;
    const int j = row_index(G, r);
    int cnt = 0;
    for (int i = 0; i + 1 < G.nx; ++i) {
        float D0 = hval(A, 0, k, r, i), D1 = hval(A, 0, k, r, i + 1);
        if ((D0 >= 0.f) == (D1 >= 0.f)) continue;
        if (!(hval(A, 4, k, r, i) > 0.5f && hval(A, 4, k, r, i + 1) > 0.5f)) continue;
        if (cnt >= KC) { atomicOr(A.err, DeviceErrors::OVERFLOW); break; }
        float t = D0 / (D0 - D1);
        auto L = [t](float a, float b) { return a + t * (b - a); };
        float Dx = L(grad_x(A, 0, k, r, i, ihx), grad_x(A, 0, k, r, i + 1, ihx));
        float Dt = L(grad_t(A, 0, k, r, i, idth), grad_t(A, 0, k, r, i + 1, idth));
        float Tx = L(grad_x(A, 1, k, r, i, ihx), grad_x(A, 1, k, r, i + 1, ihx));
        float Tt = L(grad_t(A, 1, k, r, i, idth), grad_t(A, 1, k, r, i + 1, idth));
        float thc = L(hval(A, 1, k, r, i), hval(A, 1, k, r, i + 1));
        float th0 = hval(A, 2, k, r, i), tl0 = hval(A, 3, k, r, i);
        float th1 = hval(A, 2, k, r, i + 1), tl1 = hval(A, 3, k, r, i + 1);
        float tau_hi = th0, tau_lo = tl0 + t * ((th1 - th0) + (tl1 - tl0));
        int64_t o0 = ((int64_t)r * G.nth + k) * G.nx + i;
        float Vx = L(A.V[o0], A.V[o0 + 1]), Vz = L(A.V[A.vt + o0], A.V[A.vt + o0 + 1]);
        float v = L(A.V[2 * A.vt + o0], A.V[2 * A.vt + o0 + 1]);
        float pdx = L(A.V[3 * A.vt + o0], A.V[3 * A.vt + o0 + 1]);
        float rho = L(A.rho[(int64_t)j * G.nx + i], A.rho[(int64_t)j * G.nx + i + 1]);
        float ss, cs;
        sincosf(thc, &ss, &cs);
        SrcVel sv = source_velocity(as, ss, cs);
        float gsz = sv.Vz / sv.Vn;
        float det = Dx * Tt - Dt * Tx;
        float pxl = sth / v;
        float vth = cth * Vx - sth * Vz;
        float dpx_dth = (cth * v - sth * vth) / (v * v);
        float wj = fabsf(Tt * Dx - Tx * Dt) / fabsf(Dx);
        float qx1 = 0.f, qt1 = 0.f, qx2 = 0.f, qt2 = 0.f;
        if (A.drt) {
            qx1 = L(hval(A, 5, k, r, i), hval(A, 5, k, r, i + 1));
            qt1 = L(hval(A, 6, k, r, i), hval(A, 6, k, r, i + 1));
            qx2 = L(hval(A, 7, k, r, i), hval(A, 7, k, r, i + 1));
            qt2 = L(hval(A, 8, k, r, i), hval(A, 8, k, r, i + 1));
            wj = 1.f / fabsf(qt2);  // |det J2| / |D_x| in terms of the advected families
        }
        float wreal = G.dth * wj * c_ref * c_ref / (4.f * 3.14159265358979f * sv.v * sv.v);
        float r0 = 1.f / gsz;
        int64_t slot = slot0 + cnt;
        A.pos[slot] = (float)((double)i * G.hx) + t * hx;
        A.px[slot] = pxl;
        for (int w = 0; w < A.n_omega; ++w) {
            double om = A.omega[w];
            float omf = (float)om;
            float kap = 2.f * sv.Vn / (omf * A.w0 * A.w0);
            // (dx, dtheta) = J2^-1 (r0, i kap), J2 = [[D_x, D_theta], [vartheta_x, vartheta_theta]]
            cfz dx = {Tt * r0 / det, -Dt * kap / det};
            cfz dth = {-Tx * r0 / det, Dx * kap / det};
            if (A.drt) {  // Q1 + kappa Q2 (Eq. 21 advected)
                dx = cfz{qx1, kap * qx2};
                dth = cfz{qt1, kap * qt2};
            }
            cfz dpx = {pxl * pdx * dx.re + dpx_dth * dth.re, pxl * pdx * dx.im + dpx_dth * dth.im};
            cfz M = zdiv(dpx, dx);
            cfz J = {dx.re * Vz, dx.im * Vz};
            // KMAH index 1: sigma = -1 once arg J < -1e-3 (J starts near the positive real axis)
            float sigma = atan2f(J.im, J.re) < -1e-3f ? -1.f : 1.f;
            cfz amp = zsqrt(zdiv(cfz{rho_s * sv.Vn / rho, 0.f}, J));
            cfz coef = {-wreal * sigma * amp.im, wreal * sigma * amp.re};  // i wreal sigma amp
            float ohi = omf, olo = (float)(om - (double)ohi);
            float ph = zphase(ohi, olo, tau_hi, tau_lo, A.C1, A.C2, A.C3);
            float sp, cp;
            sincosf(ph, &sp, &cp);
            cfz E = zmul(coef, cfz{cp, sp});
            if (!(isfinite(E.re) && isfinite(E.im) && isfinite(M.re) && isfinite(M.im))) {
                E = cfz{0.f, 0.f};
                M = cfz{0.f, 0.f};
            }
            A.dat[(int64_t)w * total + slot] = make_float4(E.re, E.im, M.re, fmaxf(M.im, 0.f));
        }
        ++cnt;
    }
    A.cnt[line] = cnt;
}

// One receiver per thread on the rows the branch owns (r >= r_first).
__global__ void k_zm_sum(SupArgsZ A, int r_first, float2 *u, int nz) {
    const Geom &G = A.G;
    int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y + r_first;
    if (i >= G.nx || r >= G.nr) return;
    float xr = (float)((double)i * G.hx);
    const int64_t total = (int64_t)G.nr * G.nth * KC;
    const int j = row_index(G, r);
    for (int w = 0; w < A.n_omega; ++w) {
        float om = (float)A.omega[w];
        float are = 0.f, aim = 0.f;
        for (int k = 0; k < G.nth; ++k) {
            int64_t line = (int64_t)r * G.nth + k;
            int n = A.cnt[line];
            for (int q = 0; q < n; ++q) {
                int64_t s = line * KC + q;
                float d = xr - A.pos[s];
                float4 c = A.dat[(int64_t)w * total + s];
                float dec = -0.5f * om * c.w * d * d;
                if (dec < -60.f) continue;
                float mag = __expf(dec);
                float sp, cp;
                sincosf(om * (A.px[s] * d + 0.5f * c.z * d * d), &sp, &cp);
                are += mag * (c.x * cp - c.y * sp);
                aim += mag * (c.x * sp + c.y * cp);
            }
        }
        u[((int64_t)w * nz + j) * G.nx + i] = make_float2(are, aim);
    }
}

constexpr int KMAX_Z = 32;

__global__ void k_zm_arrivals(SupArgsZ A, int r_first, uint8_t *count, double *T, float *Aout, int kmax) {
    const Geom &G = A.G;
    __shared__ float as[21];
    if (threadIdx.x < 21) as[threadIdx.x] = A.src[threadIdx.x];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y + r_first;
    if (i >= G.nx || r >= G.nr) return;
    const int j = row_index(G, r);
    const float rho_s = A.src[21], c_ref = A.src[22];
    const float rho_r = A.rho[(int64_t)j * G.nx + i];
    const float idth = 1.f / G.dth;
    const float pi8 = 25.1327412287183459f;
    double Td[KMAX_Z];
    float Al[KMAX_Z];
    int n = 0, total = 0;
    auto acell = [&](int k) {
        int64_t o = ((int64_t)r * G.nth + k) * G.nx + i;
        float vr = A.V[2 * A.vt + o];
        float thl = hval(A, 1, k, r, i);
        float ss, cs;
        sincosf(thl, &ss, &cs);
        SrcVel sv = source_velocity(as, ss, cs);
        if (A.drt) {  // point-source family: J_t = |dx_2 Vz|, A = c^2 sqrt(rho_s/rho_r) / (v_s sqrt(8 pi J_t))
            float Jt = fabsf(hval(A, 7, k, r, i) * A.V[A.vt + o]);
            return c_ref * c_ref * sqrtf(rho_s / rho_r) / (sv.v * sqrtf(pi8 * Jt));
        }
        float Dt = grad_t(A, 0, k, r, i, idth);
        return c_ref * c_ref * sqrtf(rho_s / rho_r) / (vr * sqrtf(pi8 * fabsf(sv.Vz) * fabsf(Dt)));
    };
    for (int k = 0; k + 1 < G.nth; ++k) {
        float D0 = hval(A, 0, k, r, i), D1 = hval(A, 0, k + 1, r, i);
        if ((D0 >= 0.f) == (D1 >= 0.f)) continue;
        if (!(hval(A, 4, k, r, i) > 0.5f && hval(A, 4, k + 1, r, i) > 0.5f)) continue;
        ++total;
        float t = D0 / (D0 - D1);
        float h0 = hval(A, 2, k, r, i), l0 = hval(A, 3, k, r, i);
        float h1 = hval(A, 2, k + 1, r, i), l1 = hval(A, 3, k + 1, r, i);
        double Tv = (double)h0 + ((double)l0 + (double)t * ((double)(h1 - h0) + (double)(l1 - l0)));
        float a0 = acell(k), a1 = acell(k + 1);
        float Av = a0 + t * (a1 - a0);
        int pos = n;
        while (pos > 0 && Td[pos - 1] > Tv) --pos;
        if (pos < kmax) {
            int last = n < kmax ? n : kmax - 1;
            for (int q = last; q > pos; --q) { Td[q] = Td[q - 1]; Al[q] = Al[q - 1]; }
            Td[pos] = Tv;
            Al[pos] = Av;
            if (n < kmax) ++n;
        }
    }
    if (total > kmax) atomicOr(A.err, DeviceErrors::OVERFLOW);
    int64_t node = (int64_t)j * G.nx + i;
    if (count) count[node] = (uint8_t)n;
    for (int q = 0; q < kmax; ++q) {
        if (T) T[node * kmax + q] = q < n ? Td[q] : 0.0;
        if (Aout) Aout[node * kmax + q] = q < n ? Al[q] : 0.f;
    }
}

__global__ void k_zm_source(Medium m, double xs, double zs, float *src) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double fx = (xs - m.ox) / m.hx, fz = (zs - m.oz) / m.hz;
    int ix = (int)floor(fx), iz = (int)floor(fz);
    ix = ix < 0 ? 0 : (ix > m.nx - 2 ? m.nx - 2 : ix);
    iz = iz < 0 ? 0 : (iz > m.nz - 2 ? m.nz - 2 : iz);
    double tx = fx - ix, tz = fz - iz;
    int nodes = m.nx * m.nz, n00 = iz * m.nx + ix;
    auto interp = [&](const float *f) {
        return (float)((1 - tz) * ((1 - tx) * f[n00] + tx * f[n00 + 1]) +
                       tz * ((1 - tx) * f[n00 + m.nx] + tx * f[n00 + m.nx + 1]));
    };
    float as[21];
    for (int q = 0; q < 21; ++q) as[q] = interp(m.a + (int64_t)q * nodes);
    for (int q = 0; q < 21; ++q) src[q] = as[q];
    src[21] = interp(m.rho);
    src[22] = source_velocity(as, 0.f, 1.f).v;
    src[23] = 0.f;
}

}  // namespace zm

using namespace zm;

static void split_2pi(float &C1, float &C2, float &C3) {
    const double two_pi = 6.283185307179586476925286766559;
    auto trunc_bits = [](double x, int bits) {
        int e;
        double mnt = frexp(x, &e);
        double scl = ldexp(1.0, bits);
        return ldexp(floor(mnt * scl) / scl, e);
    };
    double c1 = trunc_bits(two_pi, 15);
    double c2 = trunc_bits(two_pi - c1, 15);
    C1 = (float)c1;
    C2 = (float)c2;
    C3 = (float)(two_pi - c1 - c2);
}

size_t zmarch_device_bytes(const ZmParams &P, int nx, int nz) {
    // both branches are resident at once: nz - js rows downward and js + 1 upward
    size_t nr = (size_t)nz + 1;
    size_t cells = nr * P.n_theta * nx;
    const size_t nf = P.drt ? NF_DRT : NF_LABELS;
    size_t b = cells * 4 * (3 + 4 + nf + (P.drt ? 4 : 0));       // coefficients, velocities, history, J
    b += (size_t)2 * 3 * nf * P.n_theta * nx * 4;                 // march buffers of both branches
    b += nr * P.n_theta * (4 + (size_t)KC * (8 + 16 * P.n_omega)); // beam-centre lists
    return b + (1 << 20);
}

// Both branches of the depth march and their superposition, enqueued on s.  Outputs are device
// pointers (any may be null).  Returns the first CUDA error; device-detected errors are latched in
// d_err.  Synchronises s once per branch (to size the substeps from the largest CFL rate).
cudaError_t zmarch_run(const Medium &m, const ZmParams &P, const double *omega_dev, float2 *u,
                       uint8_t *count, double *T, float *Aout, int kmax, unsigned *d_err,
                       cudaStream_t st, egb_zmarch_info *info) {
    const int nx = m.nx, nz = m.nz, nth = P.n_theta;
    cudaError_t e = cudaSuccess;
    egb_zmarch_info stats;
    memset(&stats, 0, sizeof stats);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    auto lap = [&](int a, int b) {
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return (double)ms;
    };
    float *src = nullptr, *rate = nullptr;
    std::vector<void *> bufs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) bufs.push_back(p);
        return p;
    };
    src = (float *)alloc(32 * 4);
    rate = (float *)alloc(4);
    float c_ref = 0.f;  // source phase velocity along +z (scales the tau WENO epsilon)
    if (e == cudaSuccess) {
        zm::k_zm_source<<<1, 32, 0, st>>>(m, P.xs, P.zs, src);
        stats.kernel_launches += 1;
        e = cudaMemcpyAsync(&c_ref, src + 22, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && !(c_ref > 0.f)) c_ref = 1.f;  // non-PD medium: reported by the caller
    }
    float C1, C2, C3;
    split_2pi(C1, C2, C3);
    // Phase 1, per branch: phase angles, characteristic tables, substep count, initial data.
    struct Branch {
        bool on = false;
        int s = 1, nr = 0, n_sub = 0, nf = NF_LABELS;
        Geom G;
        int64_t plane = 0, T3 = 0;
        float2 *sc = nullptr;
        double *theta = nullptr;
        float *C = nullptr, *V = nullptr, *H = nullptr, *Jt = nullptr, *S[3] = {nullptr, nullptr, nullptr};
        int *cnt = nullptr;
        float *pos = nullptr, *px = nullptr;
        float4 *dat = nullptr;
        StageArgs A;
        float *cur = nullptr, *oa = nullptr, *ob = nullptr;
    } br[2];
    const double dth = 2.0 * P.theta_max / nth;
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        Branch &B = br[b];
        B.s = b == 0 ? 1 : -1;
        B.nr = B.s > 0 ? nz - P.js : P.js + 1;
        if (B.s < 0 && B.nr < 2) continue;  // no row above the source
        B.on = true;
        B.nf = P.drt ? NF_DRT : NF_LABELS;
        std::vector<double> th(nth);
        std::vector<float2> schost(nth);
        for (int k = 0; k < nth; ++k) {  // double on the host, then sin / cos rounded to float
            th[k] = -P.theta_max + (k + 0.5) * dth + (B.s > 0 ? 0.0 : M_PI);
            schost[k] = make_float2((float)sin(th[k]), (float)cos(th[k]));
        }
        B.sc = (float2 *)alloc((size_t)nth * 8);
        B.theta = (double *)alloc((size_t)nth * 8);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.theta, th.data(), (size_t)nth * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.sc, schost.data(), (size_t)nth * 8, cudaMemcpyHostToDevice, st);
        Geom &G = B.G;
        G.nx = nx; G.nth = nth; G.nr = B.nr; G.js = P.js; G.s = B.s;
        G.hx = m.hx; G.hz = m.hz; G.ox = m.ox; G.xs = P.xs;
        G.dth = (float)dth;
        B.plane = (int64_t)nth * nx;
        B.T3 = (int64_t)B.nr * B.plane;
        B.C = (float *)alloc((size_t)3 * B.T3 * 4);
        B.V = (float *)alloc((size_t)4 * B.T3 * 4);
        B.H = (float *)alloc((size_t)B.nf * B.T3 * 4);
        for (auto &x : B.S) x = (float *)alloc((size_t)B.nf * B.plane * 4);
        B.Jt = P.drt ? (float *)alloc((size_t)4 * B.T3 * 4) : nullptr;
        B.cnt = (int *)alloc((size_t)B.nr * nth * 4);
        B.pos = (float *)alloc((size_t)B.nr * nth * KC * 4);
        B.px = (float *)alloc((size_t)B.nr * nth * KC * 4);
        B.dat = (float4 *)alloc((size_t)P.n_omega * B.nr * nth * KC * 16 + 16);
        if (e == cudaSuccess) e = cudaMemsetAsync(rate, 0, 4, st);
        if (e != cudaSuccess) break;
        k_zm_coef<<<dim3((nx + 127) / 128, B.nr), 128, 0, st>>>(m, G, B.sc, B.C, B.V, rate, d_err);
        if (P.drt) k_zm_jac<<<dim3((nx + 127) / 128, B.nr, nth), 128, 0, st>>>(G, B.C, B.Jt);
        float hrate = 0.f;
        e = cudaMemcpyAsync(&hrate, rate, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        int n_sub = (int)std::ceil(m.hz * (double)hrate / P.cfl);
        if (!(n_sub >= 1)) n_sub = 1;
        if (n_sub > 4096) n_sub = 4096;  // a branch flagged invalid still terminates
        B.n_sub = n_sub;
        stats.n_sub[b] = n_sub;
        stats.rows[b] = B.nr;
        stats.cell_updates += (uint64_t)(B.nr - 1) * n_sub * nth * nx;
        stats.stage_passes += (uint64_t)3 * (B.nr - 1) * n_sub;
        stats.kernel_launches += 2 + (P.drt ? 1 : 0);
        const int64_t hk = (int64_t)B.nr * nx;  // history floats per angle
        k_zm_init<<<dim3((nx + 127) / 128, nth), 128, 0, st>>>(G, B.sc, B.theta, src, B.nf, B.S[0], B.H, B.T3, hk);
        StageArgs &A = B.A;
        A.G = G;
        A.ihx = (float)(1.0 / m.hx);
        A.idth = (float)(1.0 / dth);
        A.h = (float)(m.hz / n_sub);
        double h = std::max(m.hx, m.hz);
        A.eps[0] = (float)(1e-6 * h * h);
        A.eps[1] = (float)(1e-6 * dth * dth);
        A.eps[2] = (float)(1e-6 * (h / c_ref) * (h / c_ref));
        A.eps[3] = 1e-6f;
        A.cst = B.T3;
        // Q fields' scales: dx_1 ~ 1, dtheta_1 ~ 1/h, dx_2 ~ h per radian, dtheta_2 ~ 1
        A.qeps[0] = 1e-6f;
        A.qeps[1] = (float)(1e-6 / (h * h));
        A.qeps[2] = (float)(1e-6 * h * h);
        A.qeps[3] = 1e-6f;
        A.j0 = A.j1 = nullptr;
        A.hfield = B.T3;
        A.hk = hk;
        B.cur = B.S[0]; B.oa = B.S[1]; B.ob = B.S[2];
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    // Phase 2: the march.  Row interval r of every branch that has one; branches with the same
    // substep count advance together, one launch per stage for both.
    const int rmax = std::max(br[0].on ? br[0].nr - 1 : 0, br[1].on ? br[1].nr - 1 : 0);
    const bool fuse = br[0].on && br[1].on && br[0].n_sub == br[1].n_sub;
    // stage launches overlap the previous stage's last wave (programmatic dependent launch)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    auto launch = [&](int stage, Branch *b0, Branch *b1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((nx + 127) / 128, nth, b1 ? 2 : 1);
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        const StageArgs &a0 = b0->A, &a1 = b1 ? b1->A : b0->A;
        cudaError_t le;
        if (P.drt) {
            if (stage == 1) le = cudaLaunchKernelEx(&cfg, k_zm_stage<1, true>, a0, a1);
            else if (stage == 2) le = cudaLaunchKernelEx(&cfg, k_zm_stage<2, true>, a0, a1);
            else le = cudaLaunchKernelEx(&cfg, k_zm_stage<3, true>, a0, a1);
        } else {
            if (stage == 1) le = cudaLaunchKernelEx(&cfg, k_zm_stage<1, false>, a0, a1);
            else if (stage == 2) le = cudaLaunchKernelEx(&cfg, k_zm_stage<2, false>, a0, a1);
            else le = cudaLaunchKernelEx(&cfg, k_zm_stage<3, false>, a0, a1);
        }
        if (le != cudaSuccess && e == cudaSuccess) e = le;
        stats.kernel_launches += 1;
    };
    // one substep q of row interval r for the branches in list (1 or 2 of them)
    auto substep = [&](Branch **list, int n, int r, int q) {
        for (int j = 0; j < n; ++j) {
            Branch &B = *list[j];
            const double t0 = (double)q / B.n_sub;
            B.A.c0 = B.C + (int64_t)r * B.plane;
            B.A.c1 = B.C + (int64_t)(r + 1) * B.plane;
            if (P.drt) {
                B.A.j0 = B.Jt + (int64_t)r * B.plane;
                B.A.j1 = B.Jt + (int64_t)(r + 1) * B.plane;
            }
            B.A.hist = nullptr;
            B.A.in = B.cur; B.A.un = B.cur; B.A.out = B.oa; B.A.coef = 1.f; B.A.t = (float)t0;
        }
        launch(1, list[0], n > 1 ? list[1] : nullptr);
        for (int j = 0; j < n; ++j) {
            Branch &B = *list[j];
            const double t0 = (double)q / B.n_sub, dt = 1.0 / B.n_sub;
            B.A.in = B.oa; B.A.un = B.cur; B.A.out = B.ob; B.A.coef = 0.25f; B.A.t = (float)(t0 + dt);
        }
        launch(2, list[0], n > 1 ? list[1] : nullptr);
        for (int j = 0; j < n; ++j) {
            Branch &B = *list[j];
            const double t0 = (double)q / B.n_sub, dt = 1.0 / B.n_sub;
            B.A.in = B.ob; B.A.un = B.cur; B.A.out = B.oa; B.A.coef = (float)(2.0 / 3.0);
            B.A.t = (float)(t0 + 0.5 * dt);
            if (q + 1 == B.n_sub) B.A.hist = B.H + (int64_t)(r + 1) * nx;
        }
        launch(3, list[0], n > 1 ? list[1] : nullptr);
        for (int j = 0; j < n; ++j) std::swap(list[j]->cur, list[j]->oa);
    };
    if (fuse) {
        for (int r = 0; r < rmax && e == cudaSuccess; ++r) {
            Branch *list[2];
            int n = 0;
            for (auto &B : br)
                if (r + 1 < B.nr) list[n++] = &B;
            for (int q = 0; q < br[0].n_sub; ++q) substep(list, n, r, q);
            e = cudaGetLastError();
        }
    } else {
        for (auto &B : br) {
            if (!B.on) continue;
            Branch *list[1] = {&B};
            for (int r = 0; r + 1 < B.nr && e == cudaSuccess; ++r) {
                for (int q = 0; q < B.n_sub; ++q) substep(list, 1, r, q);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
    // Phase 3, per branch: beams and arrivals on the rows it owns.
    for (auto &B : br) {
        if (!B.on || e != cudaSuccess) continue;
        SupArgsZ Z;
        Z.G = B.G;
        Z.H = B.H;
        Z.hf = B.T3;
        Z.V = B.V;
        Z.vt = B.T3;
        Z.rho = m.rho;
        Z.src = src;
        Z.sc = B.sc;
        Z.cnt = B.cnt;
        Z.pos = B.pos;
        Z.px = B.px;
        Z.dat = B.dat;
        Z.n_omega = P.n_omega;
        Z.omega = omega_dev;
        Z.w0 = (float)P.w0;
        Z.C1 = C1; Z.C2 = C2; Z.C3 = C3;
        Z.err = d_err;
        Z.drt = P.drt;
        const int nr = B.nr, r_first = B.s > 0 ? 0 : 1;  // the source row belongs to the downgoing branch
        if (u && P.n_omega > 0) {
            k_zm_centres<<<(nr * nth + 127) / 128, 128, 0, st>>>(Z);
            k_zm_sum<<<dim3((nx + 127) / 128, nr - r_first), 128, 0, st>>>(Z, r_first, u, nz);
            stats.kernel_launches += 2;
        }
        if (count || T || Aout) {
            k_zm_arrivals<<<dim3((nx + 127) / 128, nr - r_first), 128, 0, st>>>(Z, r_first, count, T, Aout, kmax);
            stats.kernel_launches += 1;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    stats.setup_ms = lap(0, 1);
    stats.march_ms = lap(1, 2);
    stats.superpose_ms = lap(2, 3);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *p : bufs) cudaFree(p);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (info) *info = stats;
    return e;
}

}  // namespace egb
