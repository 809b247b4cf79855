// Gaussian-beam superposition over the source manifold and arrival extraction.
//
// Sec. 5.  Gamma = {b = 0} (Eq. 35) with b the label holding the ray's signed distance from x_s at
// closest approach; a cell counts when its labels come from the source manifold (q > 1/2) and it
// is not itself frozen.
//
//  k_beam_fields   per cell: b and the source flag                                    (Eq. 35)
//  k_centres       per grid line (row: fixed z, or column: fixed x) and angle: every sign change of
//                  b between flagged neighbours is a beam centre; its level-set gradients give the
//                  dynamic ray tracing (Eqs. 21-24) -> complex Hessian M (Eq. 25), spreading det C
//                  and amplitude (Eq. 26), weight (Eq. 33), and exp(i omega tau) with omega tau
//                  reduced mod 2 pi in double-float (Cody & Waite's split-constant reduction)
//  k_sum           per receiver: sum over angles of the beams centred on its row (offset along x:
//                  the paper's same-depth evaluation) and on its column (offset along z, for flat
//                  rays), blended by b_x^2/|grad b|^2 + b_z^2/|grad b|^2 = 1                (Eq. 34)
//  k_arrivals      per receiver: sign changes of b along theta -> traveltime and geometrical
//                  amplitude of every arrival, late arrivals included
//  k_track_branch  per cell, every BRANCH_SAMPLE steps of the evolution: the argument of the
//                  complex spreading continued through pseudo-time, which fixes the sheet of
//                  Eq. 26's square root past caustics (KMAH index)
#include "christoffel.cuh"

namespace egb {

struct SupArgs {
    Grid2D g;
    const float *st;    // padded state (u^n)
    const float *vel;   // [6][cells]
    const float *rho;   // [nz][nx]
    const float *src;   // source block
    float *B;           // [cells]
    uint8_t *FL;        // [cells]
    // beam centres: rows [nth][nz][KC], columns [nth][nx][KC]
    int *rcnt, *ccnt;
    float *rpos, *cpos, *rp, *cp;
    float4 *rdat, *cdat;  // [n_omega][line slots]: E.re, E.im, M.re, M.im
    int n_omega;
    const double *omega_dev;
    float w0;
    float iw0;              // 1 / w0: scale of the take-off family in the reference spreading
    const float *alpha;     // [cells] continued argument of the reference spreading
    const uint8_t *frozen;  // [cells] frozen source manifold
    float C1, C2, C3;     // 2 pi split for the range reduction
    unsigned *err;
};

__device__ __forceinline__ float wrap_angle(float d) {
    const float two_pi = 6.28318530717958647692f;
    return d - two_pi * rintf(d * 0.159154943091895335769f);
}

__global__ void k_beam_fields(SupArgs A) {
    const Grid2D &g = A.g;
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y, k = blockIdx.z;
    if (ix >= g.nx) return;
    int64_t p = pidx(g, k, iz, ix);
    float b = A.st[p], q = A.st[g.field + p];
    int64_t o = cidx(g, k, iz, ix);
    A.B[o] = b;
    // rays that carry source labels and have left the frozen manifold
    A.FL[o] = (q > 0.5f && !A.frozen[o]) ? 1 : 0;
}

// Gradient along x (dir 0) or z (dir 1) of a cell field F[cells], second order, one-sided at edges.
__device__ __forceinline__ float grad_line(const float *F, int64_t o, int i, int n, int64_t stride,
                                           float ih) {
    if (i == 0) return (4.f * (F[o + stride] - F[o]) - (F[o + 2 * stride] - F[o])) * 0.5f * ih;
    if (i == n - 1) return (4.f * (F[o] - F[o - stride]) - (F[o] - F[o - 2 * stride])) * 0.5f * ih;
    return (F[o + stride] - F[o - stride]) * 0.5f * ih;
}
// Same on the padded angle label, differences wrapped.
__device__ __forceinline__ float grad_line_angle(const float *F, int64_t p, int i, int n,
                                                 int64_t stride, float ih) {
    if (i == 0)
        return (4.f * wrap_angle(F[p + stride] - F[p]) - wrap_angle(F[p + 2 * stride] - F[p])) * 0.5f * ih;
    if (i == n - 1)
        return (4.f * wrap_angle(F[p] - F[p - stride]) - wrap_angle(F[p] - F[p - 2 * stride])) * 0.5f * ih;
    return wrap_angle(F[p + stride] - F[p - stride]) * 0.5f * ih;
}

struct CellData {
    float bx, bz, bt, tx, tz, tt;
    float Vx, Vz, td, pdx, pdz, v, rho, th;
    float tau_hi, tau_lo;
};

// The impact parameter is read from k_beam_fields' unpadded copy A.B, or with PADDED_B straight from
// the padded state (the same values and differences, for kernels that run without k_beam_fields).
template <bool PADDED_B = false>
__device__ CellData load_cell(const SupArgs &A, int k, int iz, int ix) {
    const Grid2D &g = A.g;
    CellData d;
    int64_t o = cidx(g, k, iz, ix);
    int64_t plane = (int64_t)g.nx * g.nz;
    float ihx = (float)(1.0 / g.hx), ihz = (float)(1.0 / g.hz), idth = (float)(1.0 / g.dth);
    int kp = (k + 1) % g.nth, km = (k - 1 + g.nth) % g.nth;
    int64_t p = pidx(g, k, iz, ix);
    if (PADDED_B) {
        d.bx = grad_line(A.st, p, ix, g.nx, 1, ihx);
        d.bz = grad_line(A.st, p, iz, g.nz, g.pitch, ihz);
        d.bt = (A.st[pidx(g, kp, iz, ix)] - A.st[pidx(g, km, iz, ix)]) * 0.5f * idth;
    } else {
        d.bx = grad_line(A.B, o, ix, g.nx, 1, ihx);
        d.bz = grad_line(A.B, o, iz, g.nz, g.nx, ihz);
        d.bt = (A.B[cidx(g, kp, iz, ix)] - A.B[cidx(g, km, iz, ix)]) * 0.5f * idth;
    }
    const float *Th = A.st + 2 * g.field;
    d.tx = grad_line_angle(Th, p, ix, g.nx, 1, ihx);
    d.tz = grad_line_angle(Th, p, iz, g.nz, g.pitch, ihz);
    d.tt = wrap_angle(Th[pidx(g, kp, iz, ix)] - Th[pidx(g, km, iz, ix)]) * 0.5f * idth;
    d.th = Th[p];
    int64_t cells = (int64_t)g.nth * plane;
    d.Vx = A.vel[o];
    d.Vz = A.vel[cells + o];
    d.td = A.vel[2 * cells + o];
    d.v = A.vel[3 * cells + o];
    d.pdx = A.vel[4 * cells + o];
    d.pdz = A.vel[5 * cells + o];
    d.rho = A.rho[(int64_t)iz * g.nx + ix];
    d.tau_hi = A.st[3 * g.field + p];
    d.tau_lo = A.st[4 * g.field + p];
    return d;
}

// Phase-space perturbations that keep the ray direction e = (Vx, Vz, thetadot) and change the
// labels (b, vartheta) by (1, 0) and (0, 1): db = (k2 x e) / D, dT = (e x k1) / D with k1 = grad b,
// k2 = grad vartheta and D = e . (k1 x k2) (the dynamic ray tracing from the level sets).  D is the
// orientation of the label coordinates (b, vartheta, tau), negative on the straight-ray data and,
// the label map being one-to-one on the source tube, negative throughout: a positive discrete D
// (under-resolved labels) is taken as -|D|, which keeps J's orientation and its argument
// continuous where the discrete D passes through zero.
__device__ __forceinline__ void ray_families(const float e[3], const float k1[3], const float k2[3],
                                             float db[3], float dT[3]) {
    float x12[3] = {k1[1] * k2[2] - k1[2] * k2[1], k1[2] * k2[0] - k1[0] * k2[2], k1[0] * k2[1] - k1[1] * k2[0]};
    float D = e[0] * x12[0] + e[1] * x12[1] + e[2] * x12[2];
    float iD = -1.f / fabsf(D);
    db[0] = (k2[1] * e[2] - k2[2] * e[1]) * iD;
    db[1] = (k2[2] * e[0] - k2[0] * e[2]) * iD;
    db[2] = (k2[0] * e[1] - k2[1] * e[0]) * iD;
    dT[0] = (e[1] * k1[2] - e[2] * k1[1]) * iD;
    dT[1] = (e[2] * k1[0] - e[0] * k1[2]) * iD;
    dT[2] = (e[0] * k1[1] - e[1] * k1[0]) * iD;
}

// Principal argument of the reference spreading J_ref = J_b + i J_T / w0 (J = dx x V of the offset
// family db and of the take-off family dT); false where the level-set Jacobian is singular.
__device__ __forceinline__ bool ref_arg(const float db[3], const float dT[3], float Vx, float Vz,
                                        float iw0, float &a) {
    float Jb = db[0] * Vz - db[1] * Vx, JT = dT[0] * Vz - dT[1] * Vx;
    if (!(isfinite(Jb) && isfinite(JT))) return false;
    a = atan2f(JT * iw0, Jb);
    return true;
}
__device__ __forceinline__ bool cell_ref_arg(float bx, float bz, float bt, float tx, float tz, float tt,
                                             float Vx, float Vz, float td, float iw0, float &a) {
    float e[3] = {Vx, Vz, td}, k1[3] = {bx, bz, bt}, k2[3] = {tx, tz, tt}, db[3], dT[3];
    ray_families(e, k1, k2, db, dT);
    return ref_arg(db, dT, Vx, Vz, iw0, a);
}
// The value a + 2 pi k (k integer) nearest to alpha.
__device__ __forceinline__ float lift_branch(float alpha, float a) {
    const float two_pi = 6.28318530717958647692f;
    return a + two_pi * rintf((alpha - a) * 0.159154943091895335769f);
}

// One sample of the continued argument on every cell of the padded state `st` (init: the initial
// data, which has no caustic, gives the principal argument; otherwise the stored value is lifted to
// the current principal argument, and kept where the level-set Jacobian is singular).  The complex
// spreading of the beam family never vanishes and the labels change continuously in pseudo-time,
// so sampled often enough this follows its argument from the straight-ray initial data to the
// steady state, which carries it onto the argument continued along the ray.
// One thread per (x, z) column and chunk of `chunk` angle planes marches through them with the
// column's b and vartheta of planes k-1, k, k+1 in registers, so a value is read from memory about
// chunk / (chunk + 2) times per cell; the x and z neighbours come through L1/L2 (neighbouring
// blocks advance nearly in step).  The chunk shrinks on small grids so that the launch still fills
// the GPU.  One launch serves up to TRACK_BATCH solves (a batch samples all its due solves at once):
// their descriptors travel in the kernel's parameter block and its blocks are numbered across them.
constexpr int TRACK_BATCH = 16;
constexpr int TRACK_THREADS = 128;
struct TrackDesc {
    Grid2D g;
    const float *st;   // padded state being sampled
    const float *vel;  // [6][cells]
    float *alpha;      // [cells]
    float iw0;
    int chunk, bx, nbx, nkc;  // planes per thread, row width, blocks along x, chunks along theta
    int block_begin;          // first block of this solve in the launch
};
struct TrackBatch {
    TrackDesc d[TRACK_BATCH];
    int n, init;
};

__global__ void __launch_bounds__(TRACK_THREADS) k_track_branch(const __grid_constant__ TrackBatch TB) {
    int i = 0;
    while (i + 1 < TB.n && (int)blockIdx.x >= TB.d[i + 1].block_begin) ++i;
    const TrackDesc &T = TB.d[i];
    const Grid2D &g = T.g;
    const int lb = (int)blockIdx.x - T.block_begin;
    const int bxi = lb % T.nbx, rest = lb / T.nbx;
    const int iz = rest % g.nz, kc = rest / g.nz;
    const int ix = bxi * T.bx + (int)threadIdx.x;
    if ((int)threadIdx.x >= T.bx || ix >= g.nx) return;
    const int k0 = kc * T.chunk, k1 = min(k0 + T.chunk, g.nth);
    const float *__restrict__ st = T.st;
    const float *__restrict__ vel = T.vel;
    float *__restrict__ alpha = T.alpha;
    float ihx = (float)(1.0 / g.hx), ihz = (float)(1.0 / g.hz), idth = (float)(1.0 / g.dth);
    const float *B = st, *Th = st + 2 * g.field;
    const int64_t p0 = pidx(g, 0, iz, ix), cells = (int64_t)g.nth * g.nx * g.nz;
    const int64_t o0 = cidx(g, 0, iz, ix), oplane = (int64_t)g.nx * g.nz;
    int kl = k0 == 0 ? g.nth - 1 : k0 - 1;
    float bm = B[p0 + kl * g.plane], tm = Th[p0 + kl * g.plane];
    float bc = B[p0 + (int64_t)k0 * g.plane], tc = Th[p0 + (int64_t)k0 * g.plane];
    for (int k = k0; k < k1; ++k) {
        int kn = k + 1 == g.nth ? 0 : k + 1;
        int64_t p = p0 + (int64_t)k * g.plane;
        float bn = B[p0 + (int64_t)kn * g.plane], tn = Th[p0 + (int64_t)kn * g.plane];
        float bx = grad_line(B, p, ix, g.nx, 1, ihx);
        float bz = grad_line(B, p, iz, g.nz, g.pitch, ihz);
        float bt = (bn - bm) * 0.5f * idth;
        float tx = grad_line_angle(Th, p, ix, g.nx, 1, ihx);
        float tz = grad_line_angle(Th, p, iz, g.nz, g.pitch, ihz);
        float tt = wrap_angle(tn - tm) * 0.5f * idth;
        int64_t o = o0 + (int64_t)k * oplane;
        float a = 0.f;
        bool ok = cell_ref_arg(bx, bz, bt, tx, tz, tt, vel[o], vel[cells + o], vel[2 * cells + o], T.iw0, a);
        if (TB.init) alpha[o] = ok ? a : 0.f;
        else if (ok) alpha[o] = lift_branch(alpha[o], a);
        bm = bc; tm = tc;
        bc = bn; tc = tn;
    }
}

cudaError_t launch_track_batch(Solve *const *sv, const float *const *st, int n, bool init, cudaStream_t s) {
    for (int i0 = 0; i0 < n; i0 += TRACK_BATCH) {
        TrackBatch TB;
        TB.n = n - i0 < TRACK_BATCH ? n - i0 : TRACK_BATCH;
        TB.init = init ? 1 : 0;
        int64_t blocks = 0;
        for (int j = 0; j < TB.n; ++j) {
            const Solve &v = *sv[i0 + j];
            const Grid2D &g = v.g;
            TrackDesc &T = TB.d[j];
            T.g = g;
            T.st = st[i0 + j];
            T.vel = v.vel;
            T.alpha = v.alpha;
            T.iw0 = (float)(1.0 / v.w0);
            // planes per thread: 32, halved while the solve would have fewer than 2^18 threads
            // (about one full wave of 152 SMs x 2048), down to 2; rows of up to 128 threads
            T.bx = g.nx >= TRACK_THREADS ? TRACK_THREADS : ((g.nx + 31) / 32) * 32;
            T.chunk = 32;
            while (T.chunk > 2 && (int64_t)g.nx * g.nz * ((g.nth + T.chunk - 1) / T.chunk) < (1 << 18)) T.chunk /= 2;
            T.nbx = (g.nx + T.bx - 1) / T.bx;
            T.nkc = (g.nth + T.chunk - 1) / T.chunk;
            T.block_begin = (int)blocks;
            blocks += (int64_t)T.nbx * g.nz * T.nkc;
        }
        if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
        if (blocks > 0) k_track_branch<<<(unsigned)blocks, TRACK_THREADS, 0, s>>>(TB);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_track_branch(const Solve &sv, const float *st, bool init, cudaStream_t s) {
    Solve *one[1] = {const_cast<Solve *>(&sv)};
    const float *sts[1] = {st};
    return launch_track_batch(one, sts, 1, init, s);
}

struct cf { float re, im; };
__device__ __forceinline__ cf cmul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
    float d = 1.f / (b.re * b.re + b.im * b.im);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
__device__ __forceinline__ cf csqrt_pr(cf z) {  // principal branch
    float r = hypotf(z.re, z.im);
    float re = sqrtf(fmaxf(0.5f * (r + z.re), 0.f));
    float im = copysignf(sqrtf(fmaxf(0.5f * (r - z.re), 0.f)), z.im);
    return {re, im};
}

// omega * tau mod 2 pi with tau = hi + lo, omega = ohi + olo (double-float), Cody-Waite reduction.
__device__ __forceinline__ float phase_mod(float ohi, float olo, float thi, float tlo, float C1,
                                           float C2, float C3) {
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

// One line (row if ROW, else column) per thread; up to KC beam centres.
// Beam data of the centre between cells i and i + 1 of a grid line (the sign change of b there):
// position, slowness along the line and, per frequency, the complex amplitude and Hessian.
template <bool ROW>
__device__ void centre_data(const SupArgs &A, const float *as, int k, int line, int i, int64_t slot,
                            int64_t lines_total) {
    const Grid2D &g = A.g;
    float rho_s = A.src[21], c_ref = A.src[22];
    // sin, cos theta_k from the source block (the float rounding of the double sin, cos of 2 pi k / n)
    const float sth = A.src[src_sc(g.nth, k)], cth = A.src[src_sc(g.nth, k) + 1];
    float h = ROW ? (float)g.hx : (float)g.hz;
    int iz0 = ROW ? line : i, ix0 = ROW ? i : line;
    int iz1 = ROW ? line : i + 1, ix1 = ROW ? i + 1 : line;
    int64_t o0 = cidx(g, k, iz0, ix0), o1 = cidx(g, k, iz1, ix1);
    float b0 = A.B[o0], b1 = A.B[o1];
    float t = b0 / (b0 - b1);
    CellData c0 = load_cell(A, k, iz0, ix0), c1 = load_cell(A, k, iz1, ix1);
    auto L = [t](float a, float b) { return a + t * (b - a); };
    float bx = L(c0.bx, c1.bx), bz = L(c0.bz, c1.bz), bt = L(c0.bt, c1.bt);
    float tx = L(c0.tx, c1.tx), tz = L(c0.tz, c1.tz), tt = L(c0.tt, c1.tt);
    float Vx = L(c0.Vx, c1.Vx), Vz = L(c0.Vz, c1.Vz), td = L(c0.td, c1.td);
    float pdx = L(c0.pdx, c1.pdx), pdz = L(c0.pdz, c1.pdz), v = L(c0.v, c1.v);
    float rho = L(c0.rho, c1.rho);
    float thc = c0.th + t * wrap_angle(c1.th - c0.th);
    float tau_hi = c0.tau_hi;
    float tau_lo = c0.tau_lo + t * ((c1.tau_hi - c0.tau_hi) + (c1.tau_lo - c0.tau_lo));
    // dynamic ray tracing from the label gradients
    float e[3] = {Vx, Vz, td}, k1[3] = {bx, bz, bt}, k2[3] = {tx, tz, tt}, db[3], dT[3];
    ray_families(e, k1, k2, db, dT);
    // sheet of the square root: the continued argument, sampled once more on both cells and
    // interpolated, against the principal argument of the reference spreading at the centre
    float al0 = A.alpha[o0], al1 = A.alpha[o1], a0, a1, ac;
    if (cell_ref_arg(c0.bx, c0.bz, c0.bt, c0.tx, c0.tz, c0.tt, c0.Vx, c0.Vz, c0.td, A.iw0, a0))
        al0 = lift_branch(al0, a0);
    if (cell_ref_arg(c1.bx, c1.bz, c1.bt, c1.tx, c1.tz, c1.tt, c1.Vx, c1.Vz, c1.td, A.iw0, a1))
        al1 = lift_branch(al1, a1);
    float sigma = 1.f;
    if (ref_arg(db, dT, Vx, Vz, A.iw0, ac)) {
        float kk = rintf((L(al0, al1) - ac) * 0.159154943091895335769f);
        sigma = (((int)kk) & 1) ? -1.f : 1.f;
    }
    float ss, cs;
    sincosf(thc, &ss, &cs);
    SrcVel sv = source_velocity(as, ss, cs);
    float pxl = sth / v, pzl = cth / v;
    float vth = cth * Vx - sth * Vz;
    float iv2 = 1.f / (v * v);
    float dpth_x = (cth * v - sth * vth) * iv2, dpth_z = (-sth * v - cth * vth) * iv2;
    // take-off measure times the row/column blend b_l^2 / |grad b|^2 (bounded where the level
    // line of b runs along the grid line): |vartheta_theta b_l - vartheta_l b_theta| |b_l| / |grad b|^2
    float g2 = bx * bx + bz * bz;
    float wj, pl, pos;
    if (ROW) {
        wj = fabsf(tt * bx - tx * bt) * fabsf(bx) / g2;
        pl = pxl;
    } else {
        wj = fabsf(tt * bz - tz * bt) * fabsf(bz) / g2;
        pl = pzl;
    }
    pos = (float)((double)i * h) + t * h;
    float wreal = g.dth * wj * c_ref * c_ref / (4.f * 3.14159265358979f * sv.v * sv.v);
    (ROW ? A.rpos : A.cpos)[slot] = pos;
    (ROW ? A.rp : A.cp)[slot] = pl;
    for (int w = 0; w < A.n_omega; ++w) {
        double om = A.omega_dev[w];
        float omf = (float)om;
        float kap = 2.f * sv.Vn / (omf * A.w0 * A.w0);
        cf dx = {db[0], kap * dT[0]}, dz = {db[1], kap * dT[1]}, dth = {db[2], kap * dT[2]};
        cf pdd = {pdx * dx.re + pdz * dz.re, pdx * dx.im + pdz * dz.im};
        cf dpx = {pxl * pdd.re + dpth_x * dth.re, pxl * pdd.im + dpth_x * dth.im};
        cf dpz = {pzl * pdd.re + dpth_z * dth.re, pzl * pdd.im + dpth_z * dth.im};
        cf J = {dx.re * Vz - dz.re * Vx, dx.im * Vz - dz.im * Vx};
        cf M;
        if (ROW) M = cdiv(cf{dpx.re * Vz - pdx * dz.re, dpx.im * Vz - pdx * dz.im}, J);
        else M = cdiv(cf{-dpz.re * Vx + pdz * dx.re, -dpz.im * Vx + pdz * dx.im}, J);
        // square root continued along the ray: J = J_b + kappa J_T has the sign of Im J_ref, so
        // the sheet found for J_ref is this frequency's too
        cf amp = csqrt_pr(cdiv(cf{rho_s * sv.Vn / rho, 0.f}, J));
        // coef = i * wreal * sigma * amp
        cf coef = {-wreal * sigma * amp.im, wreal * sigma * amp.re};
        float ohi = omf, olo = (float)(om - (double)ohi);
        float ph = phase_mod(ohi, olo, tau_hi, tau_lo, A.C1, A.C2, A.C3);
        float sp, cp;
        sincosf(ph, &sp, &cp);
        cf E = cmul(coef, cf{cp, sp});
        // a centre where the level-set Jacobian is singular (no finite beam) carries no weight
        if (!(isfinite(E.re) && isfinite(E.im) && isfinite(M.re) && isfinite(M.im))) {
            E = cf{0.f, 0.f};
            M = cf{0.f, 0.f};
        }
        // Im M annihilates V, so Im M_ll >= 0 along a grid line up to discretisation error; the
        // Gaussian factor uses max(Im M_ll, 0) so that no beam grows away from its centre
        (ROW ? A.rdat : A.cdat)[(int64_t)w * lines_total + slot] =
            make_float4(E.re, E.im, M.re, fmaxf(M.im, 0.f));
    }
}

// Beam centres of grid lines: one warp per line (k, row or column).  The lanes test 32 neighbouring
// cell pairs at a time for a sign change of b between flagged cells, a ballot numbers the
// crossings in line order, and the first KC of them are then computed one per lane (centre_data);
// more than KC set the overflow flag.  The kept centres and their order are those of a serial scan.
constexpr int CENTRE_WARPS = 4;

template <bool ROW>
__global__ void __launch_bounds__(32 * CENTRE_WARPS) k_centres(SupArgs A) {
    const Grid2D &g = A.g;
    __shared__ float as[21];
    __shared__ int at[CENTRE_WARPS][KC];
    if (threadIdx.x < 21) as[threadIdx.x] = A.src[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nl = ROW ? g.nz : g.nx;
    const int len = ROW ? g.nx : g.nz;
    const int line = blockIdx.x * CENTRE_WARPS + warp;
    const int k = blockIdx.y;
    if (line >= nl) return;  // the whole warp
    int cnt = 0;
    for (int base = 0; base + 1 < len; base += 32) {
        const int i = base + lane;
        bool cross = false;
        if (i + 1 < len) {
            int iz0 = ROW ? line : i, ix0 = ROW ? i : line;
            int iz1 = ROW ? line : i + 1, ix1 = ROW ? i + 1 : line;
            int64_t o0 = cidx(g, k, iz0, ix0), o1 = cidx(g, k, iz1, ix1);
            cross = A.FL[o0] && A.FL[o1] && ((A.B[o0] >= 0.f) != (A.B[o1] >= 0.f));
        }
        const unsigned m = __ballot_sync(0xffffffffu, cross);
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        if (cross && pos < KC) at[warp][pos] = i;
        cnt += __popc(m);
    }
    __syncwarp();
    if (cnt > KC && lane == 0) atomicOr(A.err, DeviceErrors::OVERFLOW);
    const int n = cnt < KC ? cnt : KC;
    const int64_t slot0 = ((int64_t)k * nl + line) * KC;
    const int64_t lines_total = (int64_t)g.nth * nl * KC;
    if (lane < n) centre_data<ROW>(A, as, k, line, at[warp][lane], slot0 + lane, lines_total);
    if (lane == 0) (ROW ? A.rcnt : A.ccnt)[(int64_t)k * nl + line] = n;
}

// One beam's term at a receiver offset d along its grid line (d in m), accumulated into (re, im).
__device__ __forceinline__ void beam_term(float d, float om, float p, float4 q, float &re, float &im) {
    float ph = om * (p * d + 0.5f * q.z * d * d);
    float dec = -0.5f * om * q.w * d * d;
    if (dec < -60.f) return;
    float mag = __expf(dec);
    float sp, cp;
    sincosf(ph, &sp, &cp);
    re += mag * (q.x * cp - q.y * sp);
    im += mag * (q.x * sp + q.y * cp);
}

// Eq. 34 per receiver: the sum over angles of the beams centred on its row and its column.  The
// angles of one receiver are split over SUM_LANES lanes of a warp (lane t takes theta_k with
// k = t mod SUM_LANES), whose partial sums are reduced with butterfly shuffles; a warp serves
// 32 / SUM_LANES neighbouring receivers of one row, so the lanes of one angle read the same beam
// data (the row's beams are shared by all its receivers).
constexpr int SUM_LANES = 8;
__global__ void k_sum(SupArgs A, float2 *u) {
    const Grid2D &g = A.g;
    const int lane = threadIdx.x & 31, t = lane % SUM_LANES;
    const int ix = blockIdx.x * (blockDim.x / SUM_LANES) + threadIdx.x / SUM_LANES;
    const int iz = blockIdx.y;
    const bool rx = ix < g.nx;  // lanes past the row's end still take part in the shuffles
    const int ixc = rx ? ix : g.nx - 1;
    float xr = (float)((double)ixc * g.hx), zr = (float)((double)iz * g.hz);
    int64_t rows_total = (int64_t)g.nth * g.nz * KC, cols_total = (int64_t)g.nth * g.nx * KC;
    for (int w = 0; w < A.n_omega; ++w) {
        float om = (float)A.omega_dev[w];
        float are = 0.f, aim = 0.f;
        for (int k = t; k < g.nth; k += SUM_LANES) {
            int64_t rl = (int64_t)k * g.nz + iz;
            int nr = A.rcnt[rl];
            for (int j = 0; j < nr; ++j) {
                int64_t s = rl * KC + j;
                beam_term(xr - A.rpos[s], om, A.rp[s], A.rdat[(int64_t)w * rows_total + s], are, aim);
            }
            int64_t cl = (int64_t)k * g.nx + ixc;
            int nc = A.ccnt[cl];
            for (int j = 0; j < nc; ++j) {
                int64_t s = cl * KC + j;
                beam_term(zr - A.cpos[s], om, A.cp[s], A.cdat[(int64_t)w * cols_total + s], are, aim);
            }
        }
#pragma unroll
        for (int m = SUM_LANES / 2; m > 0; m >>= 1) {
            are += __shfl_xor_sync(0xffffffffu, are, m);
            aim += __shfl_xor_sync(0xffffffffu, aim, m);
        }
        if (rx && t == 0) u[((int64_t)w * g.nz + iz) * g.nx + ix] = make_float2(are, aim);
    }
}

// Receiver-side (reciprocal) reduction of the same labels (Eq. 34 read from the receiver): at
// receiver x0, a Gaussian beam launched back along every source-labelled ray through x0 (cells
// (x0, theta) with q > 1/2, not frozen), evaluated at x_s.  The label Jacobian at x0 carries the
// launch perturbation (dx_perp, dtheta) = (1, kappa0), kappa0 = -2 i |V0| / (omega w0^2), to the
// ray's closest approach C: db = b_perp + kappa0 b_theta, dvartheta = vartheta_perp +
// kappa0 vartheta_theta (perp along (g_z, -g_x), g the unit group direction at x0).  At C the
// reversed beam's Hessian is M = -(dp/dvartheta . (g_z, -g_x))_source dvartheta / db and its phase at
// x_s is tau + M b^2 / 2.  Im M comes from the beam's Wronskian, which the symplectic ray propagator
// keeps: Im M = 2 |V0| (dp/dtheta . (g_z, -g_x))_x0 / (omega w0^2 |db|^2) (the label Jacobian
// meets this only up to discretisation error, and near the edge of the source-ray tube its Im M can
// vanish at a small |db|, leaving an undamped term whose phase hangs on the labels' last digits).
// Amplitude sqrt(rho0 |V0| / (rho_s |V_s(vartheta)| db)) (principal root: rays without a
// caustic), weight i c0^2 / (4 pi v0^2) dtheta, and the sum rescaled by
// rho_s c_s^2 / (rho0 c0^2) to the source side's normalisation (reciprocity).
// Layout: a block serves RX_W neighbouring receivers of one row (one per lane, so every gather of a
// warp is one coalesced row segment) and its RX_WARPS warps split the angles (warp w takes theta_k
// with k = w mod RX_WARPS); each cell is read once and its terms for up to RX_MAXW frequencies are
// accumulated in registers; the warps' partial sums are added in shared memory.
constexpr int RX_W = 32, RX_WARPS = 8, RX_MAXW = 8;

__global__ void __launch_bounds__(RX_W * RX_WARPS) k_sum_receiver(SupArgs A, const float *__restrict__ med_a,
                                                                   float2 *u) {
    const Grid2D &g = A.g;
    __shared__ float as[21];
    __shared__ float ohs[RX_MAXW], ols[RX_MAXW];
    __shared__ float2 part[RX_WARPS][RX_MAXW][RX_W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 21) as[threadIdx.x] = A.src[threadIdx.x];
    const int ix = blockIdx.x * RX_W + lane;
    const int iz = blockIdx.y;
    const bool rx = ix < g.nx;
    const int ixc = rx ? ix : g.nx - 1;
    const int64_t node = (int64_t)iz * g.nx + ixc, nodes = (int64_t)g.nx * g.nz;
    float a0[21];
#pragma unroll
    for (int c = 0; c < 21; ++c) a0[c] = med_a[c * nodes + node];
    const float c0 = source_velocity(a0, 0.f, 1.f).v;  // qP phase velocity along +z at x0
    const float rho0 = A.rho[node], rho_s = A.src[21], c_s = A.src[22];
    const float four_pi = 12.5663706143591729f;
    for (int wb = 0; wb < A.n_omega; wb += RX_MAXW) {  // first frequency of this pass
        const int nw = min(RX_MAXW, A.n_omega - wb);
        __syncthreads();  // as[] loaded; the previous pass's partial sums consumed
        if (threadIdx.x < nw) {  // omega as a double-float pair (hi, lo)
            double om = A.omega_dev[wb + threadIdx.x];
            float hi = (float)om;
            ohs[threadIdx.x] = hi;
            ols[threadIdx.x] = (float)(om - (double)hi);
        }
        __syncthreads();
        float are[RX_MAXW], aim[RX_MAXW];
#pragma unroll
        for (int w = 0; w < RX_MAXW; ++w) are[w] = aim[w] = 0.f;
        for (int k = warp; k < g.nth; k += RX_WARPS) {
            // rays that carry source labels and have left the frozen manifold
            const int64_t p = pidx(g, k, iz, ixc);
            if (!(A.st[g.field + p] > 0.5f) || A.frozen[cidx(g, k, iz, ixc)]) continue;
            CellData d = load_cell<true>(A, k, iz, ixc);
            const float b = A.st[p];
            const float V0 = hypotf(d.Vx, d.Vz), gx = d.Vx / V0, gz = d.Vz / V0;
            const float b_perp = d.bx * gz - d.bz * gx, t_perp = d.tx * gz - d.tz * gx;
            float sth, cth;
            sincosf(d.th, &sth, &cth);
            const SrcVel sv = source_velocity(as, sth, cth);
            const float vs_t = sv.Vx * cth - sv.Vz * sth;
            const float iv2 = 1.f / (sv.v * sv.v);
            const float dpx = (cth * sv.v - sth * vs_t) * iv2, dpz = (-sth * sv.v - cth * vs_t) * iv2;
            const float dp_perp = (dpx * sv.Vz - dpz * sv.Vx) / sv.Vn;
            // receiver medium at the cell's own angle: dp/dtheta . (g_z, -g_x) fixes Im M through
            // the beam's Wronskian (the label Jacobian keeps it only up to discretisation error)
            const float s0 = A.src[src_sc(g.nth, k)], c0k = A.src[src_sc(g.nth, k) + 1];
            const float v0_t = d.Vx * c0k - d.Vz * s0, iv02 = 1.f / (d.v * d.v);
            const float dp0x = (c0k * d.v - s0 * v0_t) * iv02, dp0z = (-s0 * d.v - c0k * v0_t) * iv02;
            const float dp0_perp = dp0x * gz - dp0z * gx;
            const float pre = rho0 * V0 / (rho_s * sv.Vn);
            const float wgt = g.dth * c0 * c0 / (four_pi * d.v * d.v);
            const float hb2 = 0.5f * b * b;
#pragma unroll
            for (int w = 0; w < RX_MAXW; ++w) {
                if (w >= nw) break;
                const float ohi = ohs[w], olo = ols[w];
                const float kap = -2.f / (ohi * A.w0 * A.w0);  // kappa0 / (i |V0|)
                const cf db = {b_perp, kap * V0 * d.bt}, dth = {t_perp, kap * V0 * d.tt};
                const float Mre = -dp_perp * cdiv(dth, db).re;
                const float Mim = -kap * V0 * dp0_perp / (db.re * db.re + db.im * db.im);
                const float dec = -ohi * Mim * hb2;
                if (!(dec > -60.f)) continue;  // far outside the beam (or not finite)
                const cf amp = csqrt_pr(cdiv(cf{pre, 0.f}, db));
                const float ph = phase_mod(ohi, olo, d.tau_hi, d.tau_lo, A.C1, A.C2, A.C3) + ohi * Mre * hb2;
                float sp, cp;
                sincosf(ph, &sp, &cp);
                const float mag = wgt * __expf(dec);
                // i * mag * amp * exp(i ph)
                const cf e = cmul(amp, cf{cp, sp});
                if (!(isfinite(e.re) && isfinite(e.im))) continue;
                are[w] -= mag * e.im;
                aim[w] += mag * e.re;
            }
        }
#pragma unroll
        for (int w = 0; w < RX_MAXW; ++w) part[warp][w][lane] = make_float2(are[w], aim[w]);
        __syncthreads();
        // warp w' adds the RX_WARPS partial sums of frequency w' (and w' + RX_WARPS, ...)
        const float sc = rho_s * c_s * c_s / (rho0 * c0 * c0);
        for (int w = warp; w < nw; w += RX_WARPS) {
            float sre = 0.f, sim = 0.f;
#pragma unroll
            for (int q = 0; q < RX_WARPS; ++q) {
                sre += part[q][w][lane].x;
                sim += part[q][w][lane].y;
            }
            if (rx) u[((int64_t)(wb + w) * g.nz + iz) * g.nx + ix] = make_float2(sc * sre, sc * sim);
        }
    }
}

constexpr int KMAX_LIMIT = 32;

__global__ void k_arrivals(SupArgs A, uint8_t *count, double *T, float *Aout, int kmax) {
    const Grid2D &g = A.g;
    __shared__ float as[21];
    if (threadIdx.x < 21) as[threadIdx.x] = A.src[threadIdx.x];
    __syncthreads();
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iz = blockIdx.y;
    if (ix >= g.nx) return;
    float rho_s = A.src[21], c_ref = A.src[22];
    float rho_r = A.rho[(int64_t)iz * g.nx + ix];
    int64_t cells = (int64_t)g.nth * g.nx * g.nz;
    float idth = (float)(1.0 / g.dth);
    const float pi8 = 25.1327412287183459f;
    double Td[KMAX_LIMIT];
    float Al[KMAX_LIMIT];
    int n = 0, total = 0;
    auto B = [&](int k) { return A.B[cidx(g, (k + g.nth) % g.nth, iz, ix)]; };
    // the geometrical amplitude of a crossing cell, with |V_s| of the source medium at its vartheta
    // (only crossing cells need it)
    auto acell = [&](int k, float bt) {
        int64_t o = cidx(g, k, iz, ix);
        float vr = A.vel[3 * cells + o];
        float sth, cth;
        sincosf(A.st[2 * g.field + pidx(g, k, iz, ix)], &sth, &cth);
        const float vsn = source_velocity(as, sth, cth).Vn;
        return c_ref * c_ref * sqrtf(rho_s / rho_r) / (vr * sqrtf(pi8 * vsn * fabsf(bt)));
    };
    for (int k = 0; k < g.nth; ++k) {
        int kn = (k + 1) % g.nth;
        int64_t o0 = cidx(g, k, iz, ix), o1 = cidx(g, kn, iz, ix);
        if (!(A.FL[o0] && A.FL[o1])) continue;
        float b0 = A.B[o0], b1 = A.B[o1];
        if ((b0 >= 0.f) == (b1 >= 0.f)) continue;
        ++total;
        float t = b0 / (b0 - b1);
        int64_t p0 = pidx(g, k, iz, ix), p1 = pidx(g, kn, iz, ix);
        float h0 = A.st[3 * g.field + p0], l0 = A.st[4 * g.field + p0];
        float h1 = A.st[3 * g.field + p1], l1 = A.st[4 * g.field + p1];
        double Tv = (double)h0 + ((double)l0 + (double)t * ((double)(h1 - h0) + (double)(l1 - l0)));
        float bt0 = (b1 - B(k - 1)) * 0.5f * idth;
        float bt1 = (B(k + 2) - b0) * 0.5f * idth;
        float a0 = acell(k, bt0), a1 = acell(kn, bt1);
        float Av = a0 + t * (a1 - a0);
        // insert keeping ascending T (equal T: later angle after)
        int pos = n;
        while (pos > 0 && Td[pos - 1] > Tv) --pos;
        if (pos < kmax) {
            int last = n < kmax ? n : kmax - 1;
            for (int j = last; j > pos; --j) { Td[j] = Td[j - 1]; Al[j] = Al[j - 1]; }
            Td[pos] = Tv;
            Al[pos] = Av;
            if (n < kmax) ++n;
        }
    }
    if (total > kmax) atomicOr(A.err, DeviceErrors::OVERFLOW);
    int64_t node = (int64_t)iz * g.nx + ix;
    if (count) count[node] = (uint8_t)n;
    for (int j = 0; j < kmax; ++j) {
        if (T) T[node * kmax + j] = j < n ? Td[j] : 0.0;
        if (Aout) Aout[node * kmax + j] = j < n ? Al[j] : 0.f;
    }
}

size_t superpose_scratch_bytes(const Solve &sv) {
    const Grid2D &g = sv.g;
    size_t cells = (size_t)g.nth * g.nx * g.nz;
    size_t rs = (size_t)g.nth * g.nz * KC, cs = (size_t)g.nth * g.nx * KC;
    size_t no = sv.omega.size();
    size_t b = cells * (4 + 1);  // B, FL
    b = (b + 255) & ~(size_t)255;
    b += (size_t)g.nth * (g.nz + g.nx) * 4 + 256;
    b += (rs + cs) * 8 + 512;
    b += no * (rs + cs) * 16 + 512;
    b += no * 8 + 256;
    return b + 4096;  // per-buffer 256-byte alignment slack
}

static void split_two_pi(float &C1, float &C2, float &C3) {
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

static cudaError_t superpose_args(Solve &sv, unsigned *d_err, cudaStream_t s, SupArgs &A);

cudaError_t launch_superpose(Solve &sv, float2 *u_dev, uint8_t *count_dev, double *T_dev,
                             float *A_dev, int kmax, unsigned *d_err, cudaStream_t s) {
    SupArgs A;
    cudaError_t e = superpose_args(sv, d_err, s, A);
    if (e != cudaSuccess) return e;
    const Grid2D &g = sv.g;
    dim3 gb((g.nx + 127) / 128, g.nz, g.nth);
    k_beam_fields<<<gb, 128, 0, s>>>(A);
    if (u_dev) {
        k_centres<true><<<dim3((g.nz + CENTRE_WARPS - 1) / CENTRE_WARPS, g.nth), 32 * CENTRE_WARPS, 0, s>>>(A);
        k_centres<false><<<dim3((g.nx + CENTRE_WARPS - 1) / CENTRE_WARPS, g.nth), 32 * CENTRE_WARPS, 0, s>>>(A);
        k_sum<<<dim3((g.nx + 256 / SUM_LANES - 1) / (256 / SUM_LANES), g.nz), 256, 0, s>>>(A, u_dev);
    }
    if (count_dev || T_dev || A_dev)
        k_arrivals<<<dim3((g.nx + 63) / 64, g.nz), 64, 0, s>>>(A, count_dev, T_dev, A_dev, kmax);
    return cudaGetLastError();
}

cudaError_t launch_superpose_receiver(Solve &sv, float2 *u_dev, unsigned *d_err, cudaStream_t s) {
    SupArgs A;
    cudaError_t e = superpose_args(sv, d_err, s, A);
    if (e != cudaSuccess) return e;
    const Grid2D &g = sv.g;
    k_sum_receiver<<<dim3((g.nx + RX_W - 1) / RX_W, g.nz), RX_W * RX_WARPS, 0, s>>>(A, sv.m->a, u_dev);
    return cudaGetLastError();
}

// Arguments of the superposition kernels: scratch carved from the solve's superposition scratch.
static cudaError_t superpose_args(Solve &sv, unsigned *d_err, cudaStream_t s, SupArgs &A) {
    const Grid2D &g = sv.g;
    size_t cells = (size_t)g.nth * g.nx * g.nz;
    size_t rs = (size_t)g.nth * g.nz * KC, cs = (size_t)g.nth * g.nx * KC;
    size_t no = sv.omega.size();
    char *base = (char *)sv.scratch;
    auto take = [&](size_t bytes) {
        char *p = base;
        base += (bytes + 255) & ~(size_t)255;
        return (void *)p;
    };
    A.g = g;
    A.st = sv.fp64 ? sv.state[0] : sv.state[sv.cur];  // the FP64 form converts into buffer 0
    A.vel = sv.vel;
    A.rho = sv.m->rho;
    A.src = sv.src;
    A.alpha = sv.alpha;
    A.iw0 = (float)(1.0 / sv.w0);
    A.B = (float *)take(cells * 4);
    A.FL = (uint8_t *)take(cells);
    A.rcnt = (int *)take((size_t)g.nth * g.nz * 4);
    A.ccnt = (int *)take((size_t)g.nth * g.nx * 4);
    A.rpos = (float *)take(rs * 4);
    A.rp = (float *)take(rs * 4);
    A.cpos = (float *)take(cs * 4);
    A.cp = (float *)take(cs * 4);
    A.rdat = (float4 *)take(no * rs * 16);
    A.cdat = (float4 *)take(no * cs * 16);
    double *om = (double *)take(no * 8);
    if ((size_t)(base - (char *)sv.scratch) > sv.scratch_bytes) return cudaErrorInvalidValue;
    cudaMemcpyAsync(om, sv.omega.data(), no * 8, cudaMemcpyHostToDevice, s);
    A.n_omega = (int)no;
    A.omega_dev = om;
    A.w0 = (float)sv.w0;
    A.frozen = sv.frozen;
    split_two_pi(A.C1, A.C2, A.C3);
    A.err = d_err;
    return cudaSuccess;
}

}  // namespace egb

// ---------------------------------------------------------------------------------------------
// Fixed scratch for egb_superpose_noalloc.  Every GPU that loads the library reserves this array
// when this module is loaded on it (under lazy module loading: at the first launch from this file
// or the first address lookup below) and keeps it until the process exits.  Host code must not pass the
// symbol itself to a kernel (in host code it names a host-side stand-in); it asks the runtime for
// the device address once per device, with that device current, and passes that address.
// No part of it has to start at zero: each superposition kernel writes every byte it later reads.
// All calls share it, so two calls whose kernels overlap on the GPU (different streams or
// contexts on one device) race on it.
// ---------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[EGB_NOALLOC_SCRATCH_BYTES];

namespace egb {

cudaError_t noalloc_scratch(int device, void **ptr) {
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[device] = p;
    }
    *ptr = addr[device];
    return cudaSuccess;
}

}  // namespace egb
