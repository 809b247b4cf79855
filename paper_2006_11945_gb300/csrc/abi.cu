// C ABI of libegb: contexts, media and solves (declared in include/egb.h).
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "egb_internal.cuh"

using namespace egb;

struct egb_ctx : public Ctx {};

namespace {

egb_status fail(egb_ctx *c, egb_status st, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

egb_status cuda_fail(egb_ctx *c, cudaError_t e, const char *what) {
    return fail(c, EGB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

size_t free_bytes() {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    return fr;
}

// Device allocation of a medium or solve of context c.  With EGB_FAIL_ALLOC=n set in the
// environment when the context was created, the allocation after the first n fails the way
// cudaMalloc does when device memory is short (host-side fault injection for the error paths).
template <class T>
static cudaError_t ctx_malloc(Ctx *c, T **p, size_t bytes) {
    if (c->fail_alloc >= 0 && c->fail_alloc-- == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void **)p, bytes);
}

void free_solve(Solve *s) {
    for (auto &p : s->state) cudaFree(p);
    for (auto &p : s->state64) cudaFree(p);
    cudaFree(s->velp64);
    if (!s->vel_shared) cudaFree(s->vel);
    cudaFree(s->velp);
    cudaFree(s->frozen);
    cudaFree(s->gs64);
    tma_release(*s);
    cudaFree(s->src);
    cudaFree(s->alpha);
    cudaFree(s->scratch);
    delete s;
}

void free_solve3d(Solve3D *s) {
    for (auto &p : s->state) cudaFree(p);
    cudaFree(s->vel);
    cudaFree(s->frozen);
    cudaFree(s->gs64);
    cudaFree(s->src);
    cudaFree(s->scratch);
    delete s;
}

void free_medium(Medium *m) {
    for (auto &kv : m->vel_cache) cudaFree(kv.second.vel);
    cudaFree(m->a);
    cudaFree(m->dadx);
    cudaFree(m->dady);
    cudaFree(m->dadz);
    cudaFree(m->rho);
    cudaFree(m->c21);
    delete m;
}

egb_status latched(egb_ctx *c) {
    unsigned bits = 0;
    cudaError_t e = cudaMemcpyAsync(&bits, c->d_err, sizeof bits, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronisation");
    if (bits) {
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
        cudaStreamSynchronize(c->stream);
        if (bits & DeviceErrors::NOT_PD) return fail(c, EGB_E_NOT_PD, "medium not positive definite (or non-finite / non-positive density) at some node");
        if (bits & DeviceErrors::TIMEOUT) return fail(c, EGB_E_TIMEOUT, "bounded device wait expired");
        if (bits & DeviceErrors::NUMERIC) return fail(c, EGB_E_NUMERIC, "non-finite value produced");
        if (bits & DeviceErrors::OVERFLOW) return fail(c, EGB_E_ARRIVAL_OVERFLOW, "more arrivals or beam centres than the capacity");
        if (bits & DeviceErrors::PARAXIAL) return fail(c, EGB_E_INVALID, "rays of a depth-march branch turn horizontal (Vz changes sign): lower theta_max");
    }
    return EGB_OK;
}

egb_status ensure_desc(egb_ctx *c, int n) {
    if (!c->d_tail && cudaMalloc(&c->d_tail, tail_plan_bytes()) != cudaSuccess) {
        cudaGetLastError();
        c->d_tail = nullptr;
        return fail(c, EGB_E_NOMEM, "stage work split");
    }
    if (c->desc_cap >= n) return EGB_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_desc);
    c->d_desc = nullptr;
    c->desc_cap = 0;
    int cap = n < 8 ? 8 : n;
    if (cudaMalloc(&c->d_desc, (size_t)9 * cap * stage_desc_bytes()) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, EGB_E_NOMEM, "stage descriptors");
    }
    c->desc_cap = cap;
    return EGB_OK;
}

// A point source in a 3-D medium (the 3-D path of egb_source).
egb_status source3d(egb_ctx *c, uint64_t mid, Medium *m, const double xs[3], int n_omega, const double *omega,
                    double beam_width, const int n_ang[2], double r0, double R_sigma, egb_solve_id *out) {
    int nth = n_ang[0], nph = n_ang[1];
    if (nth < 2 || nth > 512 || nph < 4 || nph > 1024 || nph % 2)
        return fail(c, EGB_E_INVALID, "3-D angles: n_theta in 2..512, n_phi even in 4..1024");
    double lo[3] = {m->ox, m->oy, m->oz};
    double hi[3] = {m->ox + (m->nx - 1) * m->hx, m->oy + (m->ny - 1) * m->hy, m->oz + (m->nz - 1) * m->hz};
    for (int d = 0; d < 3; ++d)
        if (!(xs[d] >= lo[d] && xs[d] <= hi[d])) return fail(c, EGB_E_INVALID, "source outside the grid");
    DeviceGuard dg(c->device);
    egb_status pre = latched(c);
    if (pre != EGB_OK) return pre;
    Solve3D *s = new Solve3D();
    s->medium_id = mid;
    s->m = m;
    Grid3D &g = s->g;
    g.nx = m->nx; g.ny = m->ny; g.nz = m->nz; g.nth = nth; g.nph = nph;
    g.pitch = ((m->nx + 5) + 1) / 2 * 2;
    g.rows = m->ny + 4;
    g.block = (int64_t)(m->nz + 4) * g.rows * g.pitch;
    g.field = g.block * nth * nph;
    g.nodes = (int64_t)m->nx * m->ny * m->nz;
    g.hx = m->hx; g.hy = m->hy; g.hz = m->hz;
    g.ox = m->ox; g.oy = m->oy; g.oz = m->oz;
    g.dth = M_PI / nth;
    g.dph = 2.0 * M_PI / nph;
    for (int d = 0; d < 3; ++d) s->xs[d] = xs[d];
    double hmax = fmax(m->hx, fmax(m->hy, m->hz));
    s->r0 = r0 > 0 ? r0 : 2.0 * hmax;
    s->w0 = beam_width;
    s->omega.assign(omega, omega + n_omega);
    // R_Sigma = max(4 r0, min(L)/8, 2 dA r_far): the source-ray tube stays wider than two angular
    // cells at the farthest corner (dA the angular spacing)
    double Lmin = fmin((g.nx - 1) * g.hx, fmin((g.ny - 1) * g.hy, (g.nz - 1) * g.hz));
    double dA = fmax(M_PI / nth, 2.0 * M_PI / nph);
    double far2 = 0.0;
    {
        double c[3] = {xs[0], xs[1], xs[2]}, o[3] = {g.ox, g.oy, g.oz}, h[3] = {g.hx, g.hy, g.hz};
        int n[3] = {g.nx, g.ny, g.nz};
        for (int d = 0; d < 3; ++d) {
            double a = (c[d] - o[d]) * (c[d] - o[d]), b = (o[d] + (n[d] - 1) * h[d] - c[d]);
            far2 += fmax(a, b * b);
        }
    }
    s->R_sigma = R_sigma > 0 ? fmax(R_sigma, s->r0) : fmax(fmax(4.0 * s->r0, Lmin / 8.0), 2.0 * dA * sqrt(far2));
    size_t cells = (size_t)g.nodes * nth * nph;
    size_t state_b = (size_t)NF3 * g.field * 4;
    s->bytes = 3 * state_b + cells * 9 * 4 + cells + (size_t)nth * nph * 24 + 32 * 4;
    if (s->bytes + (256u << 20) > free_bytes()) {
        delete s;
        return fail(c, EGB_E_NOMEM, "solve needs %zu bytes of device memory", (size_t)(s->bytes));
    }
    cudaError_t e = cudaSuccess;
    for (auto &p : s->state)
        if (e == cudaSuccess) e = ctx_malloc(c, &p, state_b);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->vel, cells * 9 * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->frozen, cells);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->gs64, sizeof(double) * 3 * nth * nph);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->src, 32 * 4);
    if (e != cudaSuccess) { cudaGetLastError(); free_solve3d(s); return fail(c, EGB_E_NOMEM, "cudaMalloc failed for the solve"); }
    float *d_rate = nullptr;
    e = cudaMalloc(&d_rate, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_rate, 0, 4, c->stream);
    if (e == cudaSuccess) e = solve3d_setup(*s, d_rate, c->stream);
    float rate = 0, cref = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rate, d_rate, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cref, s->src + 22, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_rate);
    if (e != cudaSuccess) { free_solve3d(s); return cuda_fail(c, e, "3-D solve setup"); }
    if (!(rate > 0) || !std::isfinite(rate)) { free_solve3d(s); return fail(c, EGB_E_NUMERIC, "invalid characteristic speeds"); }
    s->max_rate = rate;
    s->c_ref = cref;
    s->dt = 0.5 / rate;
    uint64_t id = c->next_id++;
    c->solves3d[id] = s;
    m->solves++;
    *out = id;
    return EGB_OK;
}

egb_status superpose3d(egb_ctx *c, Solve3D *s, void *u_out, uint8_t *count, double *T, float *A, int kmax) {
    bool want_arr = count || T || A;
    if (want_arr && (kmax < 1 || kmax > 32)) return fail(c, EGB_E_INVALID, "kmax must be in 1..32");
    DeviceGuard dg(c->device);
    size_t need = superpose3d_scratch_bytes(*s);
    cudaError_t e = cudaSuccess;
    if (s->scratch_bytes < need) {
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_bytes = 0;
        e = cudaMalloc(&s->scratch, need);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, EGB_E_NOMEM, "superposition scratch (%zu bytes)", need); }
        s->scratch_bytes = need;
    }
    size_t nodes = (size_t)s->g.nodes;
    size_t ub = s->omega.size() * nodes * 8;
    void *du = u_out;
    uint8_t *dc = count;
    double *dT = T;
    float *dA = A;
    bool hu = u_out && !is_device_ptr(u_out), hc = count && !is_device_ptr(count);
    bool hT = T && !is_device_ptr(T), hA = A && !is_device_ptr(A);
    if (hu) e = cudaMalloc(&du, ub);
    if (e == cudaSuccess && hc) e = cudaMalloc(&dc, nodes);
    if (e == cudaSuccess && hT) e = cudaMalloc(&dT, nodes * kmax * 8);
    if (e == cudaSuccess && hA) e = cudaMalloc(&dA, nodes * kmax * 4);
    if (e == cudaSuccess) e = launch_superpose3d(*s, (float2 *)du, dc, dT, dA, kmax, c->d_err, c->stream);
    if (e == cudaSuccess && hu) e = cudaMemcpyAsync(u_out, du, ub, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hc) e = cudaMemcpyAsync(count, dc, nodes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hT) e = cudaMemcpyAsync(T, dT, nodes * kmax * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hA) e = cudaMemcpyAsync(A, dA, nodes * kmax * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && (hu || hc || hT || hA)) e = cudaStreamSynchronize(c->stream);
    if (hu) cudaFree(du);
    if (hc) cudaFree(dc);
    if (hT) cudaFree(dT);
    if (hA) cudaFree(dA);
    if (e != cudaSuccess) return cuda_fail(c, e, "superpose (3-D)");
    return EGB_OK;
}

}  // namespace

extern "C" {

egb_status egb_create(egb_ctx **out, int device, void *cuda_stream, const egb_opts *opts) {
    if (!out) return EGB_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return EGB_E_CUDA;
    }
    egb_ctx *c = new egb_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->opts = opts ? *opts : egb_opts{EGB_FP32_PHASE64, 1, 0};
    if (const char *f = std::getenv("EGB_FAIL_ALLOC")) c->fail_alloc = std::strtol(f, nullptr, 10);
    DeviceGuard dg(device);
    if (cudaMalloc(&c->d_err, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return EGB_E_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->d_err);
        delete c;
        return EGB_E_CUDA;
    }
    *out = c;
    return EGB_OK;
}

egb_status egb_destroy(egb_ctx *c) {
    if (!c) return EGB_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        DeviceGuard dg(c->device);
        cudaStreamSynchronize(c->stream);
        for (auto &kv : c->solves) free_solve(kv.second);
        for (auto &kv : c->solves3d) free_solve3d(kv.second);
        for (auto &kv : c->media) free_medium(kv.second);
        c->solves.clear();
        c->solves3d.clear();
        c->media.clear();
        cudaFree(c->d_err);
        cudaFree(c->d_desc);
        cudaFree(c->d_tail);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    }
    delete c;
    return EGB_OK;
}

const char *egb_last_error(egb_ctx *c) { return c ? c->err.c_str() : "null context"; }

egb_status egb_medium(egb_ctx *c, int dim, const int n[3], const double h[3], const double origin[3],
                      const float *c21, const float *rho, egb_medium_id *out) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    if (!n || !h || !origin || !c21 || !rho || !out) return fail(c, EGB_E_INVALID, "null argument");
    if (dim != 2 && dim != 3) return fail(c, EGB_E_INVALID, "dim must be 2 or 3");
    if (n[0] < 5 || n[2] < 5 || (dim == 3 && n[1] < 5)) return fail(c, EGB_E_INVALID, "every grid extent must be >= 5");
    if (!(h[0] > 0) || !(h[2] > 0) || (dim == 3 && !(h[1] > 0))) return fail(c, EGB_E_INVALID, "spacings must be > 0");
    DeviceGuard dg(c->device);
    Medium *m = new Medium();
    m->dim = dim;
    m->nx = n[0];
    m->nz = n[2];
    m->hx = h[0];
    m->hz = h[2];
    m->ox = origin[0];
    m->oz = origin[2];
    if (dim == 3) {
        m->ny = n[1];
        m->hy = h[1];
        m->oy = origin[1];
    }
    size_t nodes = (size_t)m->nx * m->ny * m->nz;
    m->bytes = nodes * 4 * (21 * (dim + 1) + 1);
    if (m->bytes + (64u << 20) > free_bytes()) { delete m; return fail(c, EGB_E_NOMEM, "medium needs %zu bytes", m->bytes); }
    cudaError_t e = cudaSuccess;
    e = ctx_malloc(c, &m->a, nodes * 21 * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &m->dadx, nodes * 21 * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &m->dadz, nodes * 21 * 4);
    if (e == cudaSuccess && dim == 3) e = ctx_malloc(c, &m->dady, nodes * 21 * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &m->rho, nodes * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &m->c21, nodes * 21 * 4);
    if (e != cudaSuccess) { cudaGetLastError(); free_medium(m); return fail(c, EGB_E_NOMEM, "cudaMalloc failed for the medium"); }
    const float *dc = c21, *dr = rho;
    float *tc = nullptr, *tr = nullptr;
    if (!is_device_ptr(c21)) {
        e = cudaMalloc(&tc, nodes * 21 * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tc, c21, nodes * 21 * 4, cudaMemcpyHostToDevice, c->stream);
        dc = tc;
    }
    if (e == cudaSuccess && !is_device_ptr(rho)) {
        e = cudaMalloc(&tr, nodes * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tr, rho, nodes * 4, cudaMemcpyHostToDevice, c->stream);
        dr = tr;
    }
    if (e == cudaSuccess)
        e = dim == 3 ? launch_medium_prep3d(*m, dc, dr, c->d_err, c->stream)
                     : launch_medium_prep(*m, dc, dr, c->d_err, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->c21, dc, nodes * 21 * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && (tc || tr)) e = cudaStreamSynchronize(c->stream);
    cudaFree(tc);
    cudaFree(tr);
    if (e != cudaSuccess) { free_medium(m); return cuda_fail(c, e, "medium upload"); }
    uint64_t id = c->next_id++;
    c->media[id] = m;
    *out = id;
    return EGB_OK;
}

egb_status egb_source(egb_ctx *c, egb_medium_id mid, const double xs[3], int n_omega,
                      const double *omega, double beam_width, const int n_ang[2], double r0,
                      double R_sigma, egb_solve_id *out) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->media.find(mid);
    if (it == c->media.end()) return fail(c, EGB_E_INVALID, "unknown medium id");
    if (!xs || !omega || !n_ang || !out) return fail(c, EGB_E_INVALID, "null argument");
    if (n_omega < 1 || n_omega > 64) return fail(c, EGB_E_INVALID, "n_omega must be in 1..64");
    for (int i = 0; i < n_omega; ++i)
        if (!(omega[i] > 0)) return fail(c, EGB_E_INVALID, "omega must be > 0");
    if (!(beam_width > 0)) return fail(c, EGB_E_INVALID, "beam width must be > 0");
    if (R_sigma > 0 && r0 > 0 && R_sigma < r0) return fail(c, EGB_E_INVALID, "R_sigma must be at least r0");
    if (it->second->dim == 3)
        return source3d(c, mid, it->second, xs, n_omega, omega, beam_width, n_ang, r0, R_sigma, out);
    int nth = n_ang[0];
    if (nth < 8 || nth > 4096) return fail(c, EGB_E_INVALID, "n_theta must be in 8..4096");
    Medium *m = it->second;
    double x0 = m->ox, x1 = m->ox + (m->nx - 1) * m->hx, z0 = m->oz, z1 = m->oz + (m->nz - 1) * m->hz;
    if (!(xs[0] >= x0 && xs[0] <= x1 && xs[2] >= z0 && xs[2] <= z1))
        return fail(c, EGB_E_INVALID, "source outside the grid");
    DeviceGuard dg(c->device);
    egb_status pre = latched(c);  // medium validation result
    if (pre != EGB_OK) return pre;
    Solve *s = new Solve();
    s->medium_id = mid;
    s->m = m;
    Grid2D &g = s->g;
    g.nx = m->nx;
    g.nz = m->nz;
    g.nth = nth;
    g.pitch = ((m->nx + 2 * XPAD) + 3) / 4 * 4;
    g.plane = (int64_t)(g.nz + 2 * ZPAD) * g.pitch;
    g.field = g.plane * nth;
    g.hx = m->hx;
    g.hz = m->hz;
    g.ox = m->ox;
    g.oz = m->oz;
    g.dth = 2.0 * M_PI / nth;
    s->xs = xs[0];
    s->zs = xs[2];
    s->r0 = r0 > 0 ? r0 : 2.0 * (m->hx > m->hz ? m->hx : m->hz);
    s->w0 = beam_width;
    s->wait_polls = c->opts.wait_polls > 0 ? (uint32_t)c->opts.wait_polls : 0u;
    s->omega.assign(omega, omega + n_omega);
    size_t cells = (size_t)nth * g.nx * g.nz;
    size_t state_b = (size_t)NFIELD * g.field * 4;
    s->fp64 = c->opts.precision == EGB_FP64;
    size_t velp_b = (size_t)3 * g.field * (s->fp64 ? 8 : 4);
    size_t state64_b = (size_t)4 * g.field * 8;
    auto cached = s->fp64 ? m->vel_cache.end() : m->vel_cache.find(nth);
    bool reuse = cached != m->vel_cache.end();
    s->bytes = (s->fp64 ? state_b + 3 * state64_b : 3 * state_b) + (reuse ? 0 : cells * 6 * 4) + velp_b + cells +
               cells * 4 + (24 + 4 * nth) * 4;
    if (s->bytes + (256u << 20) > free_bytes()) {
        delete s;
        return fail(c, EGB_E_NOMEM, "solve needs %zu bytes of device memory", (size_t)(s->bytes));
    }
    cudaError_t e = cudaSuccess;
    if (s->fp64) {
        e = ctx_malloc(c, &s->state[0], state_b);
        for (auto &p : s->state64)
            if (e == cudaSuccess) e = ctx_malloc(c, &p, state64_b);
        if (e == cudaSuccess) e = ctx_malloc(c, &s->velp64, velp_b);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->velp64, 0, velp_b, c->stream);
    } else {
        for (auto &p : s->state)
            if (e == cudaSuccess) e = ctx_malloc(c, &p, state_b);
        if (e == cudaSuccess) e = ctx_malloc(c, &s->velp, velp_b);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->velp, 0, velp_b, c->stream);
    }
    if (reuse) {
        s->vel = cached->second.vel;
        s->vel_shared = true;
    } else if (e == cudaSuccess) {
        e = ctx_malloc(c, &s->vel, cells * 6 * 4);
    }
    if (e == cudaSuccess) e = ctx_malloc(c, &s->frozen, cells);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->gs64, sizeof(double) * 2 * s->g.nth);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->src, (24 + 4 * nth) * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, &s->alpha, cells * 4);
    if (e != cudaSuccess) { cudaGetLastError(); free_solve(s); return fail(c, EGB_E_NOMEM, "cudaMalloc failed for the solve"); }
    if (!s->fp64) {
        e = tma_prepare(*s);
        if (e != cudaSuccess) { free_solve(s); return cuda_fail(c, e, "tensor maps of the stencil"); }
    }
    // source manifold: ball radius r0 and disc radius R_Sigma = max(4 r0, min(Lx, Lz) / 8)
    {
        double Lx = (g.nx - 1) * g.hx, Lz = (g.nz - 1) * g.hz;
        double L8 = (Lx < Lz ? Lx : Lz) / 8.0;
        s->R_sigma = R_sigma > 0 ? fmax(R_sigma, s->r0) : (4.0 * s->r0 > L8 ? 4.0 * s->r0 : L8);
    }
    float *d_rate = nullptr;
    e = cudaMalloc(&d_rate, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_rate, 0, 4, c->stream);
    if (s->fp64) {
        if (e == cudaSuccess) e = launch_source_block(*s, c->stream);
        if (e == cudaSuccess) e = fp64_setup(*s, d_rate, c->stream);
    } else if (reuse) {
        // velocities of an earlier source on this medium: only the source block and the padded copy
        if (e == cudaSuccess) e = launch_source_block(*s, c->stream);
        if (e == cudaSuccess) e = launch_velp_from_vel(*s, c->stream);
        if (e == cudaSuccess) e = launch_frozen_mask(*s, c->stream);
        if (e == cudaSuccess) e = launch_init_state(*s, c->stream);
        if (e == cudaSuccess) e = launch_zero_frozen_velocity(*s, c->stream);
    } else {
        if (e == cudaSuccess) e = launch_solve_setup(*s, c->d_err, d_rate, c->stream);
        if (e == cudaSuccess) e = launch_frozen_mask(*s, c->stream);
        if (e == cudaSuccess) e = launch_init_state(*s, c->stream);
        if (e == cudaSuccess) e = launch_zero_frozen_velocity(*s, c->stream);
    }
    // first sample of the continued spreading argument, on the initial labels
    if (e == cudaSuccess && s->fp64) e = fp64_to_fp32_state(*s, c->stream);
    if (e == cudaSuccess) e = launch_track_branch(*s, s->state[s->fp64 ? 0 : s->cur], true, c->stream);
    float rate = 0, cref = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rate, d_rate, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cref, s->src + 22, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_rate);
    if (e != cudaSuccess) { free_solve(s); return cuda_fail(c, e, "solve setup"); }
    if (reuse) rate = cached->second.rate;
    if (!(rate > 0) || !std::isfinite(rate)) { free_solve(s); return fail(c, EGB_E_NUMERIC, "invalid characteristic speeds"); }
    if (!s->fp64 && !reuse) {
        m->vel_cache[nth] = Medium::VelEntry{s->vel, rate};  // the medium owns it from now on
        s->vel_shared = true;
    }
    s->max_rate = rate;
    s->c_ref = cref;
    s->cur = 0;
    if (!s->fp64) {
        egb_status st = ensure_desc(c, 1);
        if (st != EGB_OK) { free_solve(s); return st; }
        s->dt = 0.5 / s->max_rate;
        uint64_t shape = ((uint64_t)s->g.nx << 40) ^ ((uint64_t)s->g.nz << 20) ^ (uint64_t)s->g.nth;
        auto it = c->tuned_chunk.find(shape);
        if (it != c->tuned_chunk.end()) {
            tma_set_chunk(*s, it->second);
        } else {
            e = tma_autotune(*s, c->d_desc, c->d_tail, c->d_err, c->stream);
            if (e != cudaSuccess) { free_solve(s); return cuda_fail(c, e, "stencil autotuning"); }
            c->tuned_chunk[shape] = tma_chunk(*s);
        }
    }
    uint64_t id = c->next_id++;
    c->solves[id] = s;
    m->solves++;
    *out = id;
    return EGB_OK;
}

egb_status egb_evolve(egb_ctx *c, egb_solve_id sid, int steps, double cfl) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    if (steps < 0 || !(cfl > 0) || cfl > 1) return fail(c, EGB_E_INVALID, "steps >= 0 and 0 < cfl <= 1 required");
    auto i3 = c->solves3d.find(sid);
    if (i3 != c->solves3d.end()) {
        Solve3D *s3 = i3->second;
        DeviceGuard dg(c->device);
        s3->dt = cfl / s3->max_rate;
        cudaError_t e = solve3d_evolve(*s3, steps, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "3-D evolve launch");
        s3->steps += steps;
        return EGB_OK;
    }
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    Solve *s = it->second;
    DeviceGuard dg(c->device);
    s->dt = cfl / s->max_rate;
    if (s->fp64) {
        for (int i = 0; i < steps; ++i) {
            cudaError_t e = launch_rk3_step64(*s, s->dt, c->stream);
            // sample the continued spreading argument from the FP32 rounding of the state
            if (e == cudaSuccess && (s->steps + i + 1) % BRANCH_SAMPLE == 0) {
                e = fp64_to_fp32_state(*s, c->stream);
                if (e == cudaSuccess) e = launch_track_branch(*s, s->state[0], false, c->stream);
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "evolve launch");
        }
    } else {
        egb_status st = ensure_desc(c, 1);
        if (st != EGB_OK) return st;
        Solve *one[1] = {s};
        cudaError_t e = evolve_batch(one, 1, steps, c->d_desc, c->d_tail, c->d_err, c->stream, c->cap_stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "evolve launch");
    }
    s->steps += steps;
    return EGB_OK;
}

egb_status egb_evolve_batch(egb_ctx *c, int n, const egb_solve_id *ids, const int *steps, double cfl) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    if (n < 0 || (n > 0 && (!ids || !steps))) return fail(c, EGB_E_INVALID, "bad batch arguments");
    if (!(cfl > 0) || cfl > 1) return fail(c, EGB_E_INVALID, "0 < cfl <= 1 required");
    std::vector<Solve *> sv(n);
    std::vector<int> left(n);
    for (int i = 0; i < n; ++i) {
        if (c->solves3d.count(ids[i])) return fail(c, EGB_E_INVALID, "3-D solves are advanced with egb_evolve");
        auto it = c->solves.find(ids[i]);
        if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id in batch");
        if (it->second->fp64) return fail(c, EGB_E_INVALID, "FP64-form solves cannot be batched");
        if (steps[i] < 0) return fail(c, EGB_E_INVALID, "steps must be >= 0");
        for (int j = 0; j < i; ++j)
            if (sv[j] == it->second) return fail(c, EGB_E_INVALID, "a solve appears twice in the batch");
        sv[i] = it->second;
        left[i] = steps[i];
        sv[i]->dt = cfl / sv[i]->max_rate;
    }
    DeviceGuard dg(c->device);
    egb_status st = ensure_desc(c, n);
    if (st != EGB_OK) return st;
    // advance all unfinished solves by the smallest remaining count, drop the finished, repeat
    while (true) {
        std::vector<Solve *> act;
        int m = 0;
        for (int i = 0; i < n; ++i)
            if (left[i] > 0) {
                act.push_back(sv[i]);
                m = (m == 0 || left[i] < m) ? left[i] : m;
            }
        if (act.empty()) break;
        cudaError_t e = evolve_batch(act.data(), (int)act.size(), m, c->d_desc, c->d_tail, c->d_err, c->stream, c->cap_stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "batched evolve");
        for (int i = 0; i < n; ++i)
            if (left[i] > 0) {
                left[i] -= m;
                sv[i]->steps += m;
            }
    }
    return EGB_OK;
}

egb_status egb_superpose(egb_ctx *c, egb_solve_id sid, void *u_out, uint8_t *count, double *T,
                         float *A, int kmax) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto i3 = c->solves3d.find(sid);
    if (i3 != c->solves3d.end()) return superpose3d(c, i3->second, u_out, count, T, A, kmax);
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    bool want_arr = count || T || A;
    if (want_arr && (kmax < 1 || kmax > 32)) return fail(c, EGB_E_INVALID, "kmax must be in 1..32");
    Solve *s = it->second;
    DeviceGuard dg(c->device);
    size_t need = superpose_scratch_bytes(*s);
    cudaError_t e = cudaSuccess;
    if (s->scratch_bytes < need) {
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_bytes = 0;
        e = cudaMalloc(&s->scratch, need);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, EGB_E_NOMEM, "superposition scratch (%zu bytes)", need); }
        s->scratch_bytes = need;
    }
    const Grid2D &g = s->g;
    size_t nodes = (size_t)g.nx * g.nz;
    size_t ub = s->omega.size() * nodes * 8;
    // outputs: device pointers are written directly, host pointers through temporaries
    void *du = u_out;
    uint8_t *dc = count;
    double *dT = T;
    float *dA = A;
    bool hu = u_out && !is_device_ptr(u_out), hc = count && !is_device_ptr(count);
    bool hT = T && !is_device_ptr(T), hA = A && !is_device_ptr(A);
    if (hu) e = cudaMalloc(&du, ub);
    if (e == cudaSuccess && hc) e = cudaMalloc(&dc, nodes);
    if (e == cudaSuccess && hT) e = cudaMalloc(&dT, nodes * kmax * 8);
    if (e == cudaSuccess && hA) e = cudaMalloc(&dA, nodes * kmax * 4);
    if (e == cudaSuccess && s->fp64) e = fp64_to_fp32_state(*s, c->stream);
    if (e == cudaSuccess)
        e = launch_superpose(*s, (float2 *)du, dc, dT, dA, kmax, c->d_err, c->stream);
    if (e == cudaSuccess && hu) e = cudaMemcpyAsync(u_out, du, ub, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hc) e = cudaMemcpyAsync(count, dc, nodes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hT) e = cudaMemcpyAsync(T, dT, nodes * kmax * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hA) e = cudaMemcpyAsync(A, dA, nodes * kmax * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && (hu || hc || hT || hA)) e = cudaStreamSynchronize(c->stream);
    if (hu) cudaFree(du);
    if (hc) cudaFree(dc);
    if (hT) cudaFree(dT);
    if (hA) cudaFree(dA);
    if (e != cudaSuccess) return cuda_fail(c, e, "superpose");
    return EGB_OK;
}

egb_status egb_superpose_receiver(egb_ctx *c, egb_solve_id sid, void *u_out) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->solves3d.count(sid)) return fail(c, EGB_E_INVALID, "the receiver-side reduction takes 2-D solves");
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    if (!u_out) return fail(c, EGB_E_INVALID, "u_out is required");
    Solve *s = it->second;
    if (s->omega.empty()) return fail(c, EGB_E_INVALID, "the solve has no frequencies");
    DeviceGuard dg(c->device);
    size_t need = superpose_scratch_bytes(*s);
    cudaError_t e = cudaSuccess;
    if (s->scratch_bytes < need) {
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_bytes = 0;
        e = cudaMalloc(&s->scratch, need);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, EGB_E_NOMEM, "superposition scratch (%zu bytes)", need); }
        s->scratch_bytes = need;
    }
    const Grid2D &g = s->g;
    size_t ub = s->omega.size() * (size_t)g.nx * g.nz * 8;
    void *du = u_out;
    bool hu = !is_device_ptr(u_out);
    if (hu) e = cudaMalloc(&du, ub);
    if (e == cudaSuccess && s->fp64) e = fp64_to_fp32_state(*s, c->stream);
    if (e == cudaSuccess) e = launch_superpose_receiver(*s, (float2 *)du, c->d_err, c->stream);
    if (e == cudaSuccess && hu) e = cudaMemcpyAsync(u_out, du, ub, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hu) e = cudaStreamSynchronize(c->stream);
    if (hu) cudaFree(du);
    if (e != cudaSuccess) return cuda_fail(c, e, "receiver-side superpose");
    return EGB_OK;
}

egb_status egb_superpose_noalloc(egb_ctx *c, egb_solve_id sid, void *u_out, uint8_t *count,
                                 double *T, float *A, int kmax) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->solves3d.count(sid)) return fail(c, EGB_E_INVALID, "3-D solves are not accepted by egb_superpose_noalloc");
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    if ((count || T || A) && (kmax < 1 || kmax > 32)) return fail(c, EGB_E_INVALID, "kmax must be in 1..32");
    DeviceGuard dg(c->device);
    const void *outs[4] = {u_out, count, T, A};
    for (const void *p : outs)
        if (p && !is_device_ptr(p)) return fail(c, EGB_E_INVALID, "egb_superpose_noalloc needs device output pointers");
    Solve *s = it->second;
    size_t need = superpose_scratch_bytes(*s);
    if (need > EGB_NOALLOC_SCRATCH_BYTES)
        return fail(c, EGB_E_INVALID, "superposition needs %zu bytes of scratch, more than the fixed %u bytes",
                    need, (unsigned)EGB_NOALLOC_SCRATCH_BYTES);
    void *fixed = nullptr;
    cudaError_t e = noalloc_scratch(c->device, &fixed);
    if (e != cudaSuccess) return cuda_fail(c, e, "fixed scratch lookup");
    // run the ordinary superposition with the fixed array standing in for the solve's scratch
    float *own = s->scratch;
    size_t own_bytes = s->scratch_bytes;
    s->scratch = (float *)fixed;
    s->scratch_bytes = EGB_NOALLOC_SCRATCH_BYTES;
    // an FP64 solve is superposed from its FP32 rounding, written into the solve's own state[0]
    if (s->fp64) e = fp64_to_fp32_state(*s, c->stream);
    if (e == cudaSuccess) e = launch_superpose(*s, (float2 *)u_out, count, T, A, kmax, c->d_err, c->stream);
    s->scratch = own;
    s->scratch_bytes = own_bytes;
    if (e != cudaSuccess) return cuda_fail(c, e, "superpose (fixed scratch)");
    return EGB_OK;
}

egb_status egb_zmarch(egb_ctx *c, egb_medium_id mid, const double xs[3], int n_omega, const double *omega,
                      double beam_width, int n_theta, double theta_max, double cfl, int drt,
                      void *u_out, uint8_t *count, double *T, float *A, int kmax,
                      egb_zmarch_info *info) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->media.find(mid);
    if (it == c->media.end()) return fail(c, EGB_E_INVALID, "unknown medium id");
    Medium *m = it->second;
    if (m->dim != 2) return fail(c, EGB_E_INVALID, "the depth march takes 2-D media");
    if (!xs) return fail(c, EGB_E_INVALID, "null source");
    if (n_omega < 0 || n_omega > 64 || (n_omega > 0 && !omega)) return fail(c, EGB_E_INVALID, "n_omega must be in 0..64");
    for (int i = 0; i < n_omega; ++i)
        if (!(omega[i] > 0)) return fail(c, EGB_E_INVALID, "omega must be > 0");
    if (u_out && n_omega == 0) return fail(c, EGB_E_INVALID, "u_out given without frequencies");
    if (!(beam_width > 0)) return fail(c, EGB_E_INVALID, "beam width must be > 0");
    if (n_theta < 4 || n_theta > 4096) return fail(c, EGB_E_INVALID, "n_theta must be in 4..4096");
    if (!(theta_max > 0 && theta_max < 0.5 * M_PI)) return fail(c, EGB_E_INVALID, "theta_max must be in (0, pi/2)");
    if (!(cfl > 0 && cfl <= 1.0)) return fail(c, EGB_E_INVALID, "cfl must be in (0, 1]");
    if (drt != 0 && drt != 1) return fail(c, EGB_E_INVALID, "drt must be 0 or 1");
    bool want_arr = count || T || A;
    if (want_arr && (kmax < 1 || kmax > 32)) return fail(c, EGB_E_INVALID, "kmax must be in 1..32");
    if (m->nx < 4 || m->nz < 2) return fail(c, EGB_E_INVALID, "the depth march needs nx >= 4 and nz >= 2");
    double fz = (xs[2] - m->oz) / m->hz;
    int js = (int)std::lround(fz);
    if (!(std::fabs(fz - js) <= 1e-6) || js < 0 || js >= m->nz)
        return fail(c, EGB_E_INVALID, "the source depth must lie on a grid row");
    if (!(xs[0] >= m->ox && xs[0] <= m->ox + (m->nx - 1) * m->hx)) return fail(c, EGB_E_INVALID, "source outside the grid");
    DeviceGuard dg(c->device);
    egb_status pre = latched(c);  // medium validation result
    if (pre != EGB_OK) return pre;
    ZmParams P;
    P.xs = xs[0];
    P.zs = m->oz + js * m->hz;
    P.js = js;
    P.n_theta = n_theta;
    P.theta_max = theta_max;
    P.cfl = cfl;
    P.w0 = beam_width;
    P.n_omega = n_omega;
    P.drt = drt;
    size_t nodes = (size_t)m->nx * m->nz;
    size_t ub = (size_t)n_omega * nodes * 8;
    size_t need = zmarch_device_bytes(P, m->nx, m->nz) + ub + nodes * (1 + 12 * (size_t)kmax);
    if (need > free_bytes()) return fail(c, EGB_E_NOMEM, "depth march needs %zu bytes", need);
    cudaError_t e = cudaSuccess;
    double *om = nullptr;
    void *du = u_out;
    uint8_t *dc = count;
    double *dT = T;
    float *dA = A;
    bool hu = u_out && !is_device_ptr(u_out), hc = count && !is_device_ptr(count);
    bool hT = T && !is_device_ptr(T), hA = A && !is_device_ptr(A);
    if (n_omega > 0) e = cudaMalloc(&om, (size_t)n_omega * 8);
    if (e == cudaSuccess && n_omega > 0) e = cudaMemcpyAsync(om, omega, (size_t)n_omega * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && hu) e = cudaMalloc(&du, ub);
    if (e == cudaSuccess && hc) e = cudaMalloc(&dc, nodes);
    if (e == cudaSuccess && hT) e = cudaMalloc(&dT, nodes * kmax * 8);
    if (e == cudaSuccess && hA) e = cudaMalloc(&dA, nodes * kmax * 4);
    if (e == cudaSuccess && du) e = cudaMemsetAsync(du, 0, ub, c->stream);
    if (e == cudaSuccess) e = zmarch_run(*m, P, om, (float2 *)du, dc, dT, dA, kmax, c->d_err, c->stream, info);
    if (e == cudaSuccess && hu) e = cudaMemcpyAsync(u_out, du, ub, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hc) e = cudaMemcpyAsync(count, dc, nodes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hT) e = cudaMemcpyAsync(T, dT, nodes * kmax * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && hA) e = cudaMemcpyAsync(A, dA, nodes * kmax * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (hu) cudaFree(du);
    if (hc) cudaFree(dc);
    if (hT) cudaFree(dT);
    if (hA) cudaFree(dA);
    cudaFree(om);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(c, EGB_E_NOMEM, "depth march buffers") : cuda_fail(c, e, "depth march");
    }
    return latched(c);
}

egb_status egb_sync(egb_ctx *c) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    return latched(c);
}

egb_status egb_release(egb_ctx *c, uint64_t id) {
    if (!c) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    auto i3 = c->solves3d.find(id);
    if (i3 != c->solves3d.end()) {
        cudaStreamSynchronize(c->stream);
        i3->second->m->solves--;
        free_solve3d(i3->second);
        c->solves3d.erase(i3);
        return EGB_OK;
    }
    auto is = c->solves.find(id);
    if (is != c->solves.end()) {
        cudaStreamSynchronize(c->stream);
        is->second->m->solves--;
        free_solve(is->second);
        c->solves.erase(is);
        return EGB_OK;
    }
    auto im = c->media.find(id);
    if (im != c->media.end()) {
        if (im->second->solves > 0) return fail(c, EGB_E_BUSY, "medium still has solves");
        cudaStreamSynchronize(c->stream);
        free_medium(im->second);
        c->media.erase(im);
        return EGB_OK;
    }
    return fail(c, EGB_E_INVALID, "unknown id");
}

egb_status egb_get_solve_info(egb_ctx *c, egb_solve_id sid, egb_solve_info *out) {
    if (!c || !out) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto i3 = c->solves3d.find(sid);
    if (i3 != c->solves3d.end()) {
        Solve3D *s3 = i3->second;
        out->nx = s3->g.nx;
        out->nz = s3->g.nz;
        out->n_theta = s3->g.nth;
        out->n_omega = (int)s3->omega.size();
        out->steps_done = s3->steps;
        out->dt = s3->dt;
        out->max_rate = s3->max_rate;
        out->c_ref = s3->c_ref;
        out->cells = (uint64_t)s3->g.nodes * s3->g.nth * s3->g.nph;
        out->device_bytes = s3->bytes + s3->scratch_bytes;
        out->tile_chunk = 0;
        out->dim = 3;
        out->ny = s3->g.ny;
        out->n_phi = s3->g.nph;
        return EGB_OK;
    }
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    Solve *s = it->second;
    out->dim = 2;
    out->ny = 1;
    out->n_phi = 1;
    out->nx = s->g.nx;
    out->nz = s->g.nz;
    out->n_theta = s->g.nth;
    out->n_omega = (int)s->omega.size();
    out->steps_done = s->steps;
    out->dt = s->dt;
    out->max_rate = s->max_rate;
    out->c_ref = s->c_ref;
    out->cells = (uint64_t)s->g.nth * s->g.nx * s->g.nz;
    out->device_bytes = s->bytes + s->scratch_bytes;
    out->tile_chunk = s->fp64 ? 0 : tma_chunk(*s);
    return EGB_OK;
}

egb_status egb_read_state(egb_ctx *c, egb_solve_id sid, double *out) {
    if (!c || !out) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto i3 = c->solves3d.find(sid);
    if (i3 != c->solves3d.end()) {
        Solve3D *s3 = i3->second;
        DeviceGuard dg(c->device);
        size_t bytes = (size_t)8 * s3->g.nodes * s3->g.nth * s3->g.nph * 8;
        double *d = out;
        bool host = !is_device_ptr(out);
        cudaError_t e = cudaSuccess;
        if (host) e = cudaMalloc(&d, bytes);
        if (e == cudaSuccess) e = launch_read_state3d(*s3, d, c->stream);
        if (e == cudaSuccess && host) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (host) cudaFree(d);
        return e == cudaSuccess ? EGB_OK : cuda_fail(c, e, "read state (3-D)");
    }
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    Solve *s = it->second;
    DeviceGuard dg(c->device);
    size_t bytes = (size_t)4 * s->g.nth * s->g.nx * s->g.nz * 8;
    double *d = out;
    bool host = !is_device_ptr(out);
    cudaError_t e = cudaSuccess;
    if (host) e = cudaMalloc(&d, bytes);
    if (e == cudaSuccess) e = s->fp64 ? launch_read_state64(*s, d, c->stream) : launch_read_state(*s, d, c->stream);
    if (e == cudaSuccess && host) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (host) cudaFree(d);
    return e == cudaSuccess ? EGB_OK : cuda_fail(c, e, "read state");
}

egb_status egb_read_velocity(egb_ctx *c, egb_solve_id sid, float *out) {
    if (!c || !out) return EGB_E_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    auto i3 = c->solves3d.find(sid);
    if (i3 != c->solves3d.end()) {
        Solve3D *s3 = i3->second;
        DeviceGuard dg(c->device);
        size_t bytes = (size_t)9 * s3->g.nodes * s3->g.nth * s3->g.nph * 4;
        cudaError_t e = cudaMemcpyAsync(out, s3->vel, bytes, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        return e == cudaSuccess ? EGB_OK : cuda_fail(c, e, "read velocity (3-D)");
    }
    auto it = c->solves.find(sid);
    if (it == c->solves.end()) return fail(c, EGB_E_INVALID, "unknown solve id");
    Solve *s = it->second;
    DeviceGuard dg(c->device);
    size_t bytes = (size_t)6 * s->g.nth * s->g.nx * s->g.nz * 4;
    cudaError_t e = cudaMemcpyAsync(out, s->vel, bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EGB_OK : cuda_fail(c, e, "read velocity");
}

}  // extern "C"
