/* egb.h — C ABI of the GB300 anisotropic Eulerian Gaussian beam library (libegb.so).
 *
 * The library computes frequency-domain qP Green's functions of a point source in a 2-D or 3-D
 * anisotropic, heterogeneous elastic medium with the Eulerian Gaussian beam method of X. Huang,
 * "Eulerian Gaussian beams for high frequency wave propagation in inhomogeneous media of arbitrary
 * anisotropy" (arXiv 2006.11945).  The calls follow the paper's statement of the problem:
 *
 *   egb_medium    c_ijkl(x), rho(x)                         (Sec. 2, Eqs. 1, 4, 5)
 *   egb_source    point source x_s, frequencies, beam width (Sec. 4, Eq. 20; Eq. 24)
 *   egb_evolve    level sets advected through phase space   (Sec. 4, Eqs. 16, 19)
 *   egb_superpose Gaussian beams summed over the source manifold into u(x, omega), plus the
 *                 traveltime and amplitude of every arrival  (Sec. 5, Eqs. 25-26, 33-35)
 *   egb_zmarch    the paper's paraxial depth march (Eqs. 13-20) with its same-row superposition,
 *                 one call from medium to u and arrivals (one-way rays only)
 *
 * Conventions (apply to every call):
 *   - Status: every call returns egb_status; EGB_OK is 0.  No C++ exception crosses the ABI.
 *     egb_last_error(ctx) returns a NUL-terminated description of the last failure (owned by ctx,
 *     valid until the next call on ctx).
 *   - Asynchrony: work is enqueued on the CUDA stream given to egb_create.  Errors detected on the
 *     device (non-positive-definite medium, non-finite values, arrival overflow) are latched and
 *     returned by the next egb_sync (or by the next call that synchronises).
 *   - Pointers: array arguments may be host or device pointers (the library asks the CUDA runtime
 *     which).  Host outputs are written before the call returns; device outputs are written in
 *     stream order.
 *   - Ownership: the library owns media and solves (device resident until egb_release or
 *     egb_destroy).  The caller owns every buffer it passes.
 *   - Units: SI.  omega in rad/s, lengths in m, stiffness in Pa, density in kg/m^3.
 *   - Grids: nodes at origin + i*h, x horizontal, z down, stored z-major with x fastest
 *     (2-D: node = iz*nx + ix; 3-D: node = (iz*ny + iy)*nx + ix).  2-D phase angles
 *     theta_k = 2 pi k / n_theta from +z toward +x.  3-D phase directions
 *     n = (sin th cos ph, sin th sin ph, cos th) with polar angles at cell centres
 *     th_j = (j + 1/2) pi / n_theta and azimuths ph_k = 2 pi k / n_phi; direction cell
 *     dir = k * n_theta + j.
 *   - Threading: calls on one context are serialised by an internal mutex.
 */
#ifndef EGB_H
#define EGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EGB_OK = 0,
    EGB_E_INVALID = 1,          /* bad argument (sizes, pointers, unknown id, unsupported dim) */
    EGB_E_NOT_PD = 2,           /* stiffness not positive definite at some node */
    EGB_E_NOMEM = 3,            /* not enough free device memory (admission refusal) */
    EGB_E_CUDA = 4,             /* CUDA runtime error */
    EGB_E_TIMEOUT = 5,          /* a bounded device wait gave up */
    EGB_E_NUMERIC = 6,          /* non-finite value produced */
    EGB_E_ARRIVAL_OVERFLOW = 7, /* more arrivals (or beam centres) than the caller's capacity */
    EGB_E_BUSY = 8              /* object in use */
} egb_status;

typedef struct egb_ctx egb_ctx;
typedef uint64_t egb_medium_id;
typedef uint64_t egb_solve_id;

enum { EGB_FP32_PHASE64 = 0, EGB_FP64 = 1 };

typedef struct {
    int precision;      /* EGB_FP32_PHASE64: FP32 stencil/superposition with double-float tau and
                           phase; EGB_FP64: the plain all-FP64 form (comparison baseline) */
    int store_velocity; /* 1: characteristic velocities stored once per solve (the only mode) */
    int wait_polls;     /* bound on the polls of each wait of the stencil on its own copies into
                           shared memory (non-blocking polls about 32 ns apart);
                           0 (or negative) = the default, about 2^22 polls with back-off (seconds).
                           A wait that gives up latches EGB_E_TIMEOUT, returned by egb_sync: the
                           stage launch leaves the solve's state undefined, the context stays
                           usable.  Small values exist to exercise that path. */
} egb_opts;

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream` (a cudaStream_t; NULL for
 * the legacy default stream).  opts may be NULL (defaults: EGB_FP32_PHASE64, stored velocity).
 * Errors: EGB_E_INVALID (NULL out), EGB_E_CUDA (device cannot be selected). */
egb_status egb_create(egb_ctx **out, int device, void *cuda_stream, const egb_opts *opts);

/* Release every medium and solve of the context and the context itself. */
egb_status egb_destroy(egb_ctx *ctx);

/* Upload a medium (Sec. 2: a_ijkl = c_ijkl / rho, Eq. 5).
 *   dim      2 or 3
 *   n        {nx, ny, nz}; ny ignored for dim 2; every used extent >= 5
 *   h        {hx, hy, hz} node spacing (m, > 0); origin {ox, oy, oz} (m)
 *   c21      [nodes][21] float32 stiffness per node, Voigt upper triangle row by row
 *            (C11 C12 C13 C14 C15 C16 C22 ... C66), Pa; host or device
 *   rho      [nodes] float32 density per node (> 0), host or device
 *   out      receives the medium id
 * The device validates positive definiteness per node (6x6 Cholesky); failure is reported as
 * EGB_E_NOT_PD by the next synchronising call.  Errors: EGB_E_INVALID, EGB_E_NOMEM, EGB_E_CUDA. */
egb_status egb_medium(egb_ctx *ctx, int dim, const int n[3], const double h[3],
                      const double origin[3], const float *c21, const float *rho,
                      egb_medium_id *out);

/* Create a solve: a point source in a medium (Sec. 4, Eq. 20 initial data).
 *   xs          {x, y, z} source position (m), inside the grid
 *   n_omega     number of angular frequencies (1..64); omega[n_omega] rad/s (> 0), host memory
 *   beam_width  w0 (m, > 0): the Gaussian beams' 1/e half-width along the wavefront at the source
 *               (the complex initial data of Eq. 24)
 *   n_ang       2-D: {n_theta, unused}, phase-angle samples (8..4096); 3-D: {n_theta, n_phi}, polar
 *               samples (2..512) and azimuth samples (even, 4..1024)
 *   r0          radius (m) of the frozen source ball; <= 0 selects 2*max(hx, hz).  Cells within
 *               R_Sigma = max(4 r0, min(Lx, Lz)/8) of x_s whose ray still approaches the source are
 *               frozen too (the closest-approach manifold that replaces Eq. 20's initial plane;
 *               3-D: R_Sigma = max(4 r0, min(Lx, Ly, Lz)/8), r0 default 2*max(hx, hy, hz))
 *   R_sigma     that disc's radius (m) when > 0 (at least r0); <= 0 selects the default above.  Rays
 *               passing within R_Sigma of x_s carry source labels (the source-ray tube, twice
 *               R_Sigma wide); the receiver-side reduction needs it at least twice the beam width
 * The characteristic velocities depend on the medium and the phase angles only: in 2-D (FP32
 * precision) the first solve on a medium computes them for its angle count and later solves on the
 * same medium with the same count reuse them (the medium owns them until it is released).
 * Allocates the phase-space state (2-D about 3 x 20 + 12 bytes per cell, plus 24 for the first
 * source of a medium; 3-D about 3 x 36 + 37 bytes per cell) after checking free device
 * memory (EGB_E_NOMEM otherwise), computes the characteristic velocities (Eqs. 3-12), the time
 * step bound and the initial level sets.  Synchronises the context stream once (to read the CFL
 * bound).  Errors: EGB_E_INVALID, EGB_E_NOMEM, EGB_E_NOT_PD (medium failed validation), EGB_E_CUDA. */
egb_status egb_source(egb_ctx *ctx, egb_medium_id medium, const double xs[3], int n_omega,
                      const double *omega, double beam_width, const int n_ang[2], double r0,
                      double R_sigma, egb_solve_id *out);

/* Advance the level sets `steps` TVD-RK3 steps (HJ-WENO3 in x, z, theta; 3-D: x, y, z, theta, phi)
 * at Courant number cfl (0 < cfl <= 1); dt = cfl / max(|Vx|/hx + |Vz|/hz + |dtheta/dt|/dtheta)
 * (3-D: + |Vy|/hy + |dphi/dt|/dphi).  Steps compose: calling
 * twice with s1 and s2 equals one call with s1 + s2.  Asynchronous.  Errors: EGB_E_INVALID. */
egb_status egb_evolve(egb_ctx *ctx, egb_solve_id solve, int steps, double cfl);

/* Advance several solves of this context together: solve i by steps[i] TVD-RK3 steps at Courant
 * number cfl (same scheme as egb_evolve, results bit-identical to advancing each alone).  Each RK
 * stage is one persistent launch over the tiles of every solve still advancing; whole 3-step
 * rotations are captured into a CUDA graph and replayed.  Solves must be 2-D, use EGB_FP32_PHASE64
 * and be distinct.  Asynchronous.  Errors: EGB_E_INVALID, EGB_E_NOMEM, EGB_E_CUDA. */
egb_status egb_evolve_batch(egb_ctx *ctx, int n, const egb_solve_id *solves, const int *steps,
                            double cfl);

/* Superpose the Gaussian beams (Eqs. 25-26, 33-35) and extract arrivals.
 *   u_out   complex64 [n_omega][nodes] (interleaved re, im), or NULL
 *   count   uint8 [nodes] number of arrivals kept per node, or NULL
 *   T       float64 [nodes][kmax] traveltimes (s), ascending; unused slots 0; or NULL
 *   A       float32 [nodes][kmax] geometrical amplitudes, 2-D |u| sqrt(omega), 3-D |u|; unused 0;
 *           or NULL
 *   kmax    capacity per node (1..32) when count/T/A are given
 * 3-D: beams are centred where Gamma crosses the grid planes of constant x, y and z and evaluated
 * in those planes; a homogeneous isotropic medium gives exp(i k r)/(4 pi r).
 * Output scaling: rho_s c_ref^2 times the scalar qP Green's function, c_ref the source phase
 * velocity along +z; a homogeneous isotropic medium gives (i/4) H0^(1)(k r); phase exp(+i omega T)
 * (Eq. 2).  Nodes with more than kmax arrivals keep the kmax earliest and latch
 * EGB_E_ARRIVAL_OVERFLOW.  Errors: EGB_E_INVALID, EGB_E_CUDA. */
egb_status egb_superpose(egb_ctx *ctx, egb_solve_id solve, void *u_out, uint8_t *count, double *T,
                         float *A, int kmax);

/* The same Green's function as egb_superpose, summed from the receiver side (Eq. 34 read through
 * reciprocity: the field at x0 of the source x_s is that at x_s of a source at x0).  For every
 * receiver node x0 and every phase angle whose cell carries source labels (q > 1/2, not frozen),
 * a Gaussian beam is launched back along the ray through (x0, theta): the level-set Jacobian at x0
 * is the ray propagator to the ray's closest approach C to x_s (Sec. 4, the dynamic ray tracing of
 * Eqs. 21-24 read from the labels), which gives the beam's width and curvature there (Eq. 25), its
 * amplitude (Eq. 26) and its phase at x_s, tau + M b^2 / 2 (b the ray's offset from x_s at C);
 * Im M comes from the beam's Wronskian, which the ray propagator keeps, so every term decays away
 * from its ray even where the discrete label Jacobian is poorly conditioned.  The sum over theta
 * at x0, weighted as the source side (calibrated to (i/4) H0^(1) in a
 * homogeneous isotropic medium), is rescaled by rho_s c_s^2 / (rho0 c0^2) to egb_superpose's
 * normalisation.  Valid for arrivals without a caustic (KMAH index 0; principal square root); the
 * beams reach x_s about as wide as w(r) = w0 sqrt(1 + (2 r / (k w0^2))^2), so the source-ray tube
 * (egb_source's R_sigma) should be at least 2 w(r) for the farthest receiver.
 *   u_out  complex64 [n_omega][nz][nx], host or device
 * Errors: EGB_E_INVALID (3-D solve, unknown id, NULL u_out, no frequencies), EGB_E_NOMEM, EGB_E_CUDA. */
egb_status egb_superpose_receiver(egb_ctx *ctx, egb_solve_id solve, void *u_out);

/* Size of the fixed device scratch used by egb_superpose_noalloc (32 MiB). */
#define EGB_NOALLOC_SCRATCH_BYTES (32u << 20)

/* egb_superpose without any device allocation.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory at this point, for example a serving
 * loop whose device memory is already handed to a pool or caching allocator (a cudaMalloc outside
 * it can fail or fragment it), or a latency-critical loop that must not hit cudaMalloc/cudaFree
 * and their implicit device-wide synchronisation.
 * It computes exactly what egb_superpose computes for 2-D solves (3-D solve ids are not accepted),
 * but its work buffers live in one statically
 * sized device array of EGB_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  Restrictions:
 *   - u_out, count, T, A must be device pointers (or NULL); host pointers give EGB_E_INVALID;
 *   - a solve whose superposition needs more scratch than EGB_NOALLOC_SCRATCH_BYTES (about
 *     5 bytes per phase-space cell plus the beam-centre lists, i.e. up to a few million cells) is
 *     refused with EGB_E_INVALID and a message giving both sizes;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress with
 *     that device current); make that first call before any stream capture.  The array is taken
 *     when the library's superposition module is first loaded on the device; under the runtime's
 *     default lazy module loading that can be this first call itself (or the first egb_superpose);
 *   - a solve made in an EGB_FP64 context is superposed from the FP32 rounding of its state,
 *     written into the solve's own buffers, exactly as egb_superpose does;
 *   - every call shares the array: calls whose kernels may overlap on the GPU (other streams or
 *     other contexts on the same device) race and must be serialised by the caller.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
egb_status egb_superpose_noalloc(egb_ctx *ctx, egb_solve_id solve, void *u_out, uint8_t *count,
                                 double *T, float *A, int kmax);

/* Wait for the context stream and report latched device errors (then clear them). */
egb_status egb_sync(egb_ctx *ctx);

/* Free a medium or a solve (ids are unique across both kinds).  Errors: EGB_E_INVALID (unknown),
 * EGB_E_BUSY (a medium that still has solves). */
egb_status egb_release(egb_ctx *ctx, uint64_t id);

const char *egb_last_error(egb_ctx *ctx);

/* Read-only facts about a solve (not a step of the method; for callers that report throughput). */
typedef struct {
    int nx, nz, n_theta, n_omega;
    int steps_done;
    double dt;             /* pseudo-time step of the last egb_evolve (s) */
    double max_rate;       /* max(|Vx|/hx + |Vz|/hz + |thetadot|/dtheta) (1/s) */
    double c_ref;          /* source qP phase velocity along +z (m/s) */
    uint64_t cells;        /* nx * nz * n_theta */
    uint64_t device_bytes; /* device memory held by the solve */
    int tile_chunk;        /* theta planes per stencil work item chosen by the autotuner (0: FP64 or 3-D) */
    int dim;               /* 2 or 3 */
    int ny;                /* 3-D: nodes along y (1 in 2-D) */
    int n_phi;             /* 3-D: azimuth samples (1 in 2-D); n_theta is then the polar count */
} egb_solve_info;

egb_status egb_get_solve_info(egb_ctx *ctx, egb_solve_id solve, egb_solve_info *out);

/* Copy the level sets of a solve to the caller.  3-D: out = [8][n_phi][n_theta][nz][ny][nx] float64
 * holding bx, by, bz (offset of the ray from x_s at closest approach, m), n0x, n0y, n0z (take-off
 * phase direction), q, tau (s).  2-D: out = [4][n_theta][nz][nx] float64 holding
 * b (signed distance of the ray from x_s at closest approach, m), q (1 where the labels come from
 * the source manifold, 0 from the domain boundary), vartheta (angle label, rad), tau (s), host or
 * device.  Synchronous.  For tests and diagnostics (the state otherwise stays on the device). */
egb_status egb_read_state(egb_ctx *ctx, egb_solve_id solve, double *out);

/* Copy the characteristic velocities: out = [6][n_theta][nz][nx] float32 holding Vx, Vz,
 * dtheta/dt, v (phase velocity), dp_x/dt, dp_z/dt; 3-D: [9][n_phi][n_theta][nz][ny][nx] holding
 * Vx, Vy, Vz, dtheta/dt, dphi/dt, v, dp_x/dt, dp_y/dt, dp_z/dt.  Synchronous. */
egb_status egb_read_velocity(egb_ctx *ctx, egb_solve_id solve, float *out);

/* The paper's own formulation: the level sets marched in depth (Sec. 3-4, Eqs. 13-20) and the
 * Gaussian beams centred where each depth row crosses Gamma = {X = x_s}, evaluated along that row
 * (Sec. 5, Eqs. 25-28, 33-35).  2-D media only.  One call runs both branches from the source row:
 * downgoing rays (phase angles theta_k = -theta_max + (k + 1/2) dtheta, dtheta = 2 theta_max /
 * n_theta, from +z toward +x) fill the rows at and below the source, upgoing rays (the same angles
 * + pi) the rows above it.  Every ray of a branch must keep the sign of its vertical group velocity
 * (Eq. 13); a medium where one does not gives EGB_E_INVALID (lower theta_max).  Each row interval is
 * crossed in ceil(h_z max(|dx/dz|/h_x + |dtheta/dz|/dtheta) / cfl) TVD-RK3 substeps.
 *   medium     a 2-D medium id (validated: a non positive definite medium gives EGB_E_NOT_PD)
 *   xs         source (x, y, z); z must lie on a grid row (within 1e-6 h_z), x anywhere on the grid
 *   omega      n_omega angular frequencies (rad/s, > 0; host pointer), 0 <= n_omega <= 64
 *   beam_width_m  w0 > 0: initial transverse beam Hessian i 2 / (omega w0^2) (Eq. 24)
 *   n_theta    angles per branch, 4..4096; theta_max in (0, pi/2); cfl in (0, 1]
 *   drt        dynamic ray tracing of the beams and arrival amplitudes: 0 from the gradients of
 *              the labels at fixed depth; 1 advected with the march (Eq. 21, read anisotropically:
 *              the ray perturbations (dx, dtheta) of the offset and take-off families obey
 *              Q_z + u Q_x + w Q_theta = J Q, J the (x, theta) Jacobian of (dx/dz, dtheta/dz); about
 *              36 more bytes per phase-space cell)
 *   u_out      complex64 [n_omega][nz][nx] (host or device), or NULL
 *   count, T, A   arrivals per node ([nz][nx] uint8, [nz][nx][kmax] float64 s, float32), each may
 *              be NULL; kmax in 1..32 when any is given; more arrivals than kmax give
 *              EGB_E_ARRIVAL_OVERFLOW after the earliest kmax are written
 *   info       optional (NULL allowed): facts about the run for callers that report throughput,
 *              not a step of the method (see egb_zmarch_info)
 * Rays entering through the grid's x edges or the ends of the angle range carry no source-plane
 * labels: an advected source indicator (ghost value 0) keeps them out of beams and arrivals.
 * Synchronous: returns when the outputs are written.  The work buffers (about 48 bytes per
 * phase-space cell of both branches together, which advance in the same launches) are allocated
 * and freed by the call; EGB_E_NOMEM when they do not fit. */
typedef struct {
    int n_sub[2];             /* TVD-RK3 substeps per row interval: [0] downgoing, [1] upgoing (0: absent) */
    int rows[2];              /* rows of each branch, the source row included */
    uint64_t cell_updates;    /* (theta, x) cells advanced one full substep, both branches */
    uint64_t stage_passes;    /* stage passes over a branch's (theta, x) plane (3 per substep and
                               * branch); branches with equal substep counts share launches */
    uint64_t kernel_launches; /* every kernel the call launched */
    double setup_ms;          /* device time of the characteristic tables (CUDA events, ctx stream) */
    double march_ms;          /* device time of the depth march (initial data and stages) */
    double superpose_ms;      /* device time of the beams and arrivals */
} egb_zmarch_info;

egb_status egb_zmarch(egb_ctx *ctx, egb_medium_id medium, const double xs[3], int n_omega,
                      const double *omega, double beam_width_m, int n_theta, double theta_max,
                      double cfl, int drt, void *u_out, uint8_t *count, double *T, float *A,
                      int kmax, egb_zmarch_info *info);

#ifdef __cplusplus
}
#endif

#endif /* EGB_H */
