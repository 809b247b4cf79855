// Internal declarations shared by the CUDA translation units of libegb (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/egb.h"

namespace egb {

// ---------------------------------------------------------------------------------------------
// Layout of the 2-D phase-space state.
// Every field is a stack of n_theta planes; a plane has (nz + 4) rows of `pitch` floats.  Row r
// holds depth index iz = r - 2 (two ghost rows on each side); column c holds ix = c - XPAD
// (XPAD = 4 keeps the interior 16-byte aligned; columns XPAD-2, XPAD-1 and XPAD+nx, XPAD+nx+1 are
// the ghost layers).  Ghosts hold the initial data permanently (Dirichlet inflow).
// Fields: 0 b (impact parameter at closest approach to the source), 1 q (source indicator),
// 2 vartheta, 3 tau_hi, 4 tau_lo (double-float tau).
// ---------------------------------------------------------------------------------------------
constexpr int XPAD = 4;
constexpr int ZPAD = 2;
constexpr int NFIELD = 5;
constexpr int KC = 16;  // beam centres kept per grid line and angle
// Steps between two samples of the continued argument of the complex spreading (the sheet of the
// amplitude's square root past caustics): a sample follows every step whose count is a multiple.
constexpr int BRANCH_SAMPLE = 9;

struct Grid2D {
    int nx, nz, nth;
    int pitch;        // floats per padded row
    int64_t plane;    // floats per padded plane = (nz + 4) * pitch
    int64_t field;    // floats per field = nth * plane
    double hx, hz, ox, oz, dth;
};

__host__ __device__ inline int64_t pidx(const Grid2D &g, int k, int iz, int ix) {
    return (int64_t)k * g.plane + (int64_t)(iz + ZPAD) * g.pitch + (ix + XPAD);
}
__host__ __device__ inline int64_t cidx(const Grid2D &g, int k, int iz, int ix) {
    return ((int64_t)k * g.nz + iz) * g.nx + ix;
}

// Voigt bookkeeping: 21 constants stored as the upper triangle of the 6x6 matrix, row by row.
__host__ __device__ constexpr int voigt(int i, int j) { return i == j ? i : 6 - i - j; }
__host__ __device__ constexpr int tri21(int I, int J) {
    return I <= J ? I * 6 - I * (I - 1) / 2 + (J - I) : J * 6 - J * (J - 1) / 2 + (I - J);
}
__host__ __device__ constexpr int aidx(int i, int j, int k, int l) {
    return tri21(voigt(i, j), voigt(k, l));
}

// Source manifold.  A phase cell is frozen at its straight-ray data when it lies in the ball
// |x - x_s| <= r0, or within R_Sigma of x_s while its ray still approaches the source
// ((x - x_s) . g_s(theta) < 0, g_s the source medium's unit group direction).  The decision is
// taken once per solve in FP64 (k_frozen) and stored as a byte mask; the stencil kernels see a
// frozen cell as one whose stored velocity copy (velp) is exactly zero.

// Double-float helpers (Knuth's TwoSum and Dekker's FastTwoSum).
struct ff { float hi, lo; };
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
// (hi, lo) + d  ->  renormalised double-float
__device__ __forceinline__ ff ff_add_f(float hi, float lo, float d) {
    ff s = two_sum(hi, d);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, lo));
}

struct DeviceErrors {  // bits latched by kernels, read by egb_sync
    enum : unsigned { NOT_PD = 1u, NUMERIC = 2u, OVERFLOW = 4u, TIMEOUT = 8u, PARAXIAL = 16u };
};

// ---------------------------------------------------------------------------------------------
// Host-side objects
// ---------------------------------------------------------------------------------------------
struct Medium {
    int nx, nz;
    double hx, hz, ox, oz;
    int dim = 2, ny = 1;    // 3-D media: ny nodes along y at spacing hy from oy
    double hy = 1.0, oy = 0.0;
    float *a = nullptr;     // [21][nz][(ny)][nx]  a = c / rho
    float *dadx = nullptr;  // [21][nz][(ny)][nx]
    float *dady = nullptr;  // [21][nz][ny][nx] (3-D only)
    float *dadz = nullptr;  // [21][nz][(ny)][nx]
    float *rho = nullptr;   // [nz][(ny)][nx]
    float *c21 = nullptr;   // [nodes][21] device copy of the input stiffness
    // characteristic velocities of the 2-D FP32 path per angle count: they depend on the medium and
    // the phase angles only, so every source on this medium shares them (owned here, freed with
    // the medium)
    struct VelEntry { float *vel; float rate; };
    std::unordered_map<int, VelEntry> vel_cache;
    int solves = 0;
    size_t bytes = 0;
};

// A solve's source block (floats, device): [0,21) a_s, [21] rho_s, [22] c_ref, [23] pad,
// [24 + 2k] psx_k, [25 + 2k] psz_k (slowness at the source), [24 + 2 nth + 2k] sin, cos theta_k
__host__ __device__ inline int src_ps(int k) { return 24 + 2 * k; }
__host__ __device__ inline int src_sc(int nth, int k) { return 24 + 2 * nth + 2 * k; }

struct Solve {
    uint64_t medium_id;
    Medium *m;
    Grid2D g;
    double xs, zs, r0, w0;
    double R_sigma;         // radius of the closest-approach manifold's disc
    uint8_t *frozen = nullptr;  // [nth][nz][nx] 1 on the frozen source manifold
    double *gs64 = nullptr;     // [nth][2] source-medium unit group direction (FP64)
    std::vector<double> omega;
    float *state[3] = {nullptr, nullptr, nullptr};  // three padded buffers of NFIELD fields
    int cur = 0;                                     // buffer holding u^n
    float *vel = nullptr;   // [6][nth][nz][nx]: Vx, Vz, thetadot, v, pdx, pdz
    bool vel_shared = false;  // vel belongs to the medium's cache
    float *velp = nullptr;  // [3][nth][nz+4][pitch]: Vx, Vz, thetadot in the padded state layout
    void *tma = nullptr;    // tensor maps of the TMA stencil
    bool fp64 = false;      // plain all-FP64 form
    double *state64[3] = {nullptr, nullptr, nullptr};  // [4 fields] Yx, Yz, vartheta, tau (FP64 form)
    double *velp64 = nullptr;                           // [3] padded Vx, Vz, thetadot (FP64 form)
    float *src = nullptr;   // source block: a_s[21], rho_s, c_ref, then [nth] x (psx, psz)
    float *alpha = nullptr; // [nth][nz][nx] continued argument of the reference complex spreading
    float *scratch = nullptr;  // superposition scratch (lazily sized)
    size_t scratch_bytes = 0;
    double max_rate = 0, dt = 0, c_ref = 0;
    int steps = 0;
    size_t bytes = 0;
    uint32_t wait_polls = 0;  // bound of the stencil's waits on its copies (0: the default)
};

// ---------------------------------------------------------------------------------------------
// 3-D phase space (x, y, z, theta, phi): n = (sin th cos ph, sin th sin ph, cos th), theta at cell
// centres th_j = (j + 1/2) pi / n_theta, phi_k = 2 pi k / n_phi (n_phi even).  A direction cell is
// dir = k * n_theta + j.  Every field is a stack of n_phi * n_theta blocks; a block is
// (nz + 4) x (ny + 4) rows of `pitch` floats with the interior at z, y offsets 2 and x offset
// XPAD3 = 2 (even, so that pairs of x-neighbours are 8-byte aligned); the two ghost layers on each
// side hold the initial data permanently.  Fields: 0-2 b (offset of the ray from x_s at closest
// approach), 3-5 n0 (take-off phase direction), 6 q (source indicator), 7 tau_hi, 8 tau_lo.
// ---------------------------------------------------------------------------------------------
constexpr int XPAD3 = 2;
constexpr int NF3 = 9;

struct Grid3D {
    int nx, ny, nz, nth, nph;
    int pitch;        // floats per padded row (even, >= nx + 5)
    int rows;         // padded rows per z slice = ny + 4
    int64_t block;    // floats per direction block = (nz + 4) * rows * pitch
    int64_t field;    // floats per field = nph * nth * block
    int64_t nodes;    // nx * ny * nz
    double hx, hy, hz, ox, oy, oz, dth, dph;
};

__host__ __device__ inline int64_t pidx3(const Grid3D &g, int dir, int iz, int iy, int ix) {
    return (int64_t)dir * g.block + ((int64_t)(iz + 2) * g.rows + (iy + 2)) * g.pitch + (ix + XPAD3);
}
__host__ __device__ inline int64_t cidx3(const Grid3D &g, int dir, int iz, int iy, int ix) {
    return (int64_t)dir * g.nodes + ((int64_t)iz * g.ny + iy) * g.nx + ix;
}

struct Solve3D {
    uint64_t medium_id;
    Medium *m;
    Grid3D g;
    double xs[3], r0, w0, R_sigma;
    std::vector<double> omega;
    float *state[3] = {nullptr, nullptr, nullptr};  // u^n, stage buffers (NF3 padded fields each)
    float *vel = nullptr;       // [9][cells]: Vx, Vy, Vz, thetadot, phidot, v, pdx, pdy, pdz
    uint8_t *frozen = nullptr;  // [cells] 1 on the frozen source manifold
    double *gs64 = nullptr;     // [dir][3] source-medium unit group direction (FP64)
    float *src = nullptr;       // a_s[21], rho_s, c_ref
    float *scratch = nullptr;   // superposition scratch
    size_t scratch_bytes = 0;
    double max_rate = 0, dt = 0, c_ref = 0;
    int steps = 0;
    size_t bytes = 0;
};

struct StageDesc;  // per-solve, per-stage descriptor of the batched stencil (liouville_tma.cu)

struct Ctx {
    int device;
    cudaStream_t stream;
    egb_opts opts;
    std::mutex mu;
    std::string err;
    uint64_t next_id = 1;
    std::unordered_map<uint64_t, Medium *> media;
    std::unordered_map<uint64_t, Solve *> solves;
    std::unordered_map<uint64_t, Solve3D *> solves3d;
    unsigned *d_err = nullptr;  // device error bits
    StageDesc *d_desc = nullptr;  // stage descriptors of batched launches (device)
    int desc_cap = 0;             // capacity in solves (9 descriptors per solve)
    void *d_tail = nullptr;       // the stage launches' tail work split (device, tail_plan_bytes())
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture CUDA graphs
    // theta chunk chosen by the stencil autotuner, per grid shape (nx, nz, n_theta): later solves
    // of the same shape reuse it instead of timing the candidates again
    std::unordered_map<uint64_t, int> tuned_chunk;
    // host-side fault injection (EGB_FAIL_ALLOC at egb_create): the number of device allocations of
    // media and solves that succeed before one fails; -1 when off
    long fail_alloc = -1;
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_medium_prep(const Medium &m, const float *c21_dev, const float *rho_dev,
                               unsigned *d_err, cudaStream_t s);
cudaError_t launch_solve_setup(const Solve &sv, unsigned *d_err, float *d_rate, cudaStream_t s);
cudaError_t launch_velp_from_vel(const Solve &sv, cudaStream_t s);
cudaError_t launch_init_state(const Solve &sv, cudaStream_t s);
cudaError_t launch_frozen_mask(const Solve &sv, cudaStream_t s);
cudaError_t launch_zero_frozen_velocity(const Solve &sv, cudaStream_t s);
cudaError_t tma_prepare(Solve &sv);
void tma_release(Solve &sv);
size_t stage_desc_bytes();
size_t tail_plan_bytes();
int tma_chunk(const Solve &sv);
void tma_set_chunk(Solve &sv, int chunk);
cudaError_t tma_autotune(Solve &sv, StageDesc *d_desc, void *d_tail, unsigned *err, cudaStream_t s);
cudaError_t evolve_batch(Solve **sv, int n, int steps, StageDesc *d_desc, void *d_tail, unsigned *err, cudaStream_t s,
                         cudaStream_t cap);
// One sample of the continued spreading argument from the padded FP32 state st (init: first sample).
cudaError_t launch_track_branch(const Solve &sv, const float *st, bool init, cudaStream_t s);
cudaError_t launch_track_batch(Solve *const *sv, const float *const *st, int n, bool init, cudaStream_t s);
cudaError_t launch_superpose(Solve &sv, float2 *u_dev, uint8_t *count_dev, double *T_dev,
                             float *A_dev, int kmax, unsigned *d_err, cudaStream_t s);
size_t superpose_scratch_bytes(const Solve &sv);
// Receiver-side (reciprocal) reduction of the solve's labels into u_dev [n_omega][nz][nx].
cudaError_t launch_superpose_receiver(Solve &sv, float2 *u_dev, unsigned *d_err, cudaStream_t s);
// Device address of the fixed superposition scratch (EGB_NOALLOC_SCRATCH_BYTES) on `device`, which
// must be the current device; looked up once per device.
cudaError_t noalloc_scratch(int device, void **ptr);
cudaError_t launch_read_state(const Solve &sv, double *out_dev, cudaStream_t s);
cudaError_t launch_source_block(const Solve &sv, cudaStream_t s);
cudaError_t fp64_setup(Solve &sv, float *d_rate, cudaStream_t s);
cudaError_t launch_rk3_step64(Solve &sv, double dt, cudaStream_t s);
cudaError_t fp64_to_fp32_state(Solve &sv, cudaStream_t s);
cudaError_t launch_read_state64(const Solve &sv, double *out_dev, cudaStream_t s);
cudaError_t launch_medium_a(int nodes, const float *c21_dev, const float *rho_dev, float *a,
                            unsigned *d_err, cudaStream_t s);

// 3-D path (solve3d.cu)
cudaError_t launch_medium_prep3d(const Medium &m, const float *c21_dev, const float *rho_dev,
                                 unsigned *d_err, cudaStream_t s);
cudaError_t solve3d_setup(Solve3D &sv, float *d_rate, cudaStream_t s);
cudaError_t solve3d_evolve(Solve3D &sv, int steps, cudaStream_t s);
size_t superpose3d_scratch_bytes(const Solve3D &sv);
cudaError_t launch_superpose3d(Solve3D &sv, float2 *u_dev, uint8_t *count_dev, double *T_dev,
                               float *A_dev, int kmax, unsigned *d_err, cudaStream_t s);
cudaError_t launch_read_state3d(const Solve3D &sv, double *out_dev, cudaStream_t s);

// Paraxial depth march (zmarch.cu): both branches from the source row and their superposition.
struct ZmParams {
    double xs, zs;      // source position (zs on grid row js)
    int js;
    int n_theta;        // angles per branch
    double theta_max;   // half-width of the angle range (rad)
    double cfl;
    double w0;          // beam width (m)
    int n_omega;
    int drt;            // 0: dynamic ray tracing from label gradients, 1: advected (Eq. 21)
};
size_t zmarch_device_bytes(const ZmParams &P, int nx, int nz);
cudaError_t zmarch_run(const Medium &m, const ZmParams &P, const double *omega_dev, float2 *u,
                       uint8_t *count, double *T, float *A, int kmax, unsigned *d_err, cudaStream_t s,
                       egb_zmarch_info *info);

}  // namespace egb
