// TMA-staged Liouville stencil (the hot loop): persistent, streaming along theta.
//
// Same scheme as the plain stage kernel (Eqs. 16, 19 in pseudo-time; third-order HJ-WENO upwinded
// by the velocity sign; Shu-Osher TVD-RK3 in increment form: u1 = u + dt L(u),
// u2 = u + 1/4 ((u1 - u) + dt L(u1)), u_new = u + 2/3 ((u2 - u) + dt L(u2)); double-float tau kept
// with an error-free sum; wrapped angle-label differences; frozen cells of the source manifold copy
// u^n; ghosts are never written), organised for GB300:
//
//  * two CTAs per SM (192 threads, under 114 KB of shared memory each) loop over work items
//    (x-tile of 64 cells, z-tile of 6 rows, theta chunk);
//  * for each theta plane a single 4-D TMA copy brings all five state fields of the tile plus its
//    x/z halo (a 72 x 10 box: x from -4 so the copy starts on a 16-byte boundary, z from -2) into a
//    ring of shared-memory slots, each starting on a 128-byte boundary; the theta stencil reads the
//    neighbouring planes' slots, so every plane is fetched from HBM once per tile and chunk;
//  * u^n (stages 2, 3) and the stored velocities of the centre plane come by a second TMA copy;
//  * mbarrier transaction counts track completion; every wait is bounded and a timeout latches
//    EGB_E_TIMEOUT, drains the copies in flight and leaves the kernel;
//  * each thread updates two neighbouring x cells with packed FP32x2 arithmetic where it maps.
#include <cuda.h>

#include "egb_internal.cuh"

namespace egb {

namespace tma {
constexpr int TX = 64, TZ = 6;                     // tile (cells)
constexpr int HX = TX + 8, HZ = TZ + 4;            // halo box (x -4..67, z -2..TZ+1)
constexpr int RING = 6, RING2 = 2;                 // plane slots, centre-plane slots
constexpr int CTAS_PER_SM = 2;                     // two CTAs resident per SM (shared memory < 114 KB each)
constexpr int TAIL_SEGS_PER_CTA = 2;               // capacity of the tail work split (segments per CTA)
constexpr int HALO_FLOATS = NFIELD * HZ * HX;      // floats one halo copy brings
constexpr int UN_FLOATS = NFIELD * TZ * TX;        // floats of the u^n copy
constexpr int V_FLOATS = 3 * TZ * TX;              // floats of the velocity copy
// every TMA destination starts on a 128-byte boundary: slots are padded to multiples of 32 floats
constexpr int pad32(int n) { return (n + 31) / 32 * 32; }
constexpr int HALO_STRIDE = pad32(HALO_FLOATS);
constexpr int UN_STRIDE = pad32(UN_FLOATS);
constexpr int SLOT2_STRIDE = UN_STRIDE + pad32(V_FLOATS);
static_assert((HALO_STRIDE * 4) % 128 == 0 && (UN_STRIDE * 4) % 128 == 0 && (SLOT2_STRIDE * 4) % 128 == 0,
              "TMA destinations must stay 128-byte aligned");
constexpr size_t SMEM_BYTES = sizeof(float) * ((size_t)RING * HALO_STRIDE + (size_t)RING2 * SLOT2_STRIDE) +
                              8 * (RING + RING2);
constexpr int THREADS = 32 * TZ;
}  // namespace tma

// One solve, one RK stage.  Lives in device memory; a launch processes the work items of several
// solves (batching), item i of solve s being item i - item_begin of that solve.
struct StageDesc {
    const CUtensorMap *mapK;  // halo map of the state being differentiated (device address)
    const CUtensorMap *mapN;  // interior map of u^n
    const CUtensorMap *mapV;  // interior map of the padded velocities
    float *out;
    Grid2D g;
    float dt, coef, ihx, ihz, idth;
    float eps[4];
    int tiles_x, tiles_z, chunk, items, item_begin;
    uint32_t polls;  // limit of each bounded wait on a copy of this solve's planes
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking poll: true once the phase with this parity has completed.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls, returning false.  The default bound (2^22 polls with
// back-off) is seconds.  A caller-set bound uses non-blocking polls 32 ns apart, so that a small
// bound gives up while a copy is still in flight.
constexpr uint32_t DEFAULT_POLLS = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, uint32_t limit = DEFAULT_POLLS) {
    if (limit >= DEFAULT_POLLS) {
        for (uint32_t i = 0; i < limit; ++i) {
            if (mbar_try_wait(b, parity)) return true;
            if (i > 16) __nanosleep(128);
        }
        return false;
    }
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_test_wait(b, parity)) return true;
        __nanosleep(32);
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// ---- packed two-cell arithmetic ------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed FMA (b * -1 + a is exactly the rounded difference)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float2 wrap2(float2 d) {
    const float two_pi = 6.28318530717958647692f;
    const float inv = 0.159154943091895335769f;
    float2 k = f2(rintf(d.x * inv), rintf(d.y * inv));
    return fma2(f2(-two_pi, -two_pi), k, d);
}

// Upwind side of two cells along one axis: flow towards + (the left-biased stencil) or towards -.
struct Up2 {
    bool lx, ly;  // cell 0 / cell 1 flows towards +
    float2 sig;   // +1 for flow towards +, -1 otherwise
};
__device__ __forceinline__ Up2 upwind2(float2 v) {
    Up2 u;
    u.lx = v.x > 0.f;
    u.ly = v.y > 0.f;
    u.sig = f2(u.lx ? 1.f : -1.f, u.ly ? 1.f : -1.f);
    return u;
}

// Third-order HJ-WENO (the scheme of Eq. 19's spatial discretisation, as in the FP64 form) for two
// cells, from the four consecutive differences d_0..d_3 of the five-point stencil, written with the
// second differences e_j = d_{j+1} - d_j.  The upwind smoothness term is e_0 (flow towards +) or
// e_2 (towards -); with A = e_up^2 + eps, B = e_1^2 + eps and w = B^2 / (B^2 + 2 A^2),
//     2 h u_x = (d_1 + d_2) + sig w (e_up - e_1),
// which is the central difference less w/2 times the upwind curvature (d_0 - 2 d_1 + d_2 towards +,
// d_3 - 2 d_2 + d_1 towards -).  Returns 2 h u_x; the caller scales by velocity / (2 h).
__device__ __forceinline__ float2 weno3_2(const float2 d[4], const Up2 &up, float2 eps2) {
    float2 e0 = sub2(d[1], d[0]), e1 = sub2(d[2], d[1]), e2 = sub2(d[3], d[2]);
    float2 E = f2(up.lx ? e0.x : e2.x, up.ly ? e0.y : e2.y);
    float2 A = fma2(E, E, eps2);
    float2 B = fma2(e1, e1, eps2);
    float2 B2 = mul2(B, B);
    float2 den = fma2(mul2(A, A), f2(2.f, 2.f), B2);
    float2 num = mul2(B2, up.sig);
    // w = num / den with one approximate reciprocal per lane and one packed multiply
    float rx, ry;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(den.y));
    float2 w = mul2(num, f2(rx, ry));
    return fma2(w, sub2(E, e1), add2(d[1], d[2]));
}

__device__ __forceinline__ float2 deriv2(const float2 s[5], const Up2 &up, float2 eps2, bool angle) {
    float2 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d[j] = sub2(s[j + 1], s[j]);
        if (angle) d[j] = wrap2(d[j]);
    }
    return weno3_2(d, up, eps2);
}

__device__ __forceinline__ float2 deriv2_ff(const float2 h[5], const float2 l[5], const Up2 &up, float2 eps2) {
    float2 d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = add2(sub2(h[j + 1], h[j]), sub2(l[j + 1], l[j]));
    return weno3_2(d, up, eps2);
}

// BOUNDED: the waits on this launch's copies use the solves' caller-set poll bound (egb_opts.wait_polls)
// instead of the default one; a separate instantiation keeps the default kernel free of it.
template <int STAGE, bool BOUNDED>
__global__ void __launch_bounds__(tma::THREADS, tma::CTAS_PER_SM)
    k_rk3_tma(const StageDesc *__restrict__ D, int nsolves, int full_items, const int4 *__restrict__ tail,
              const int *__restrict__ tail_begin, unsigned *err) {
    using namespace tma;
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring = reinterpret_cast<float *>(smem);
    float *ring2 = ring + RING * HALO_STRIDE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ring2 + RING2 * SLOT2_STRIDE);
    uint64_t *bar2 = bar + RING;
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int tx = tid & 31, tz = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < RING + RING2; ++s) mbar_init(bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    uint32_t phase = 0, phase2 = 0;      // parity bit per slot (identical in every thread)
    uint32_t pending = 0, pending2 = 0;  // slots with a copy in flight (thread 0 only)
    const uint32_t bytes_halo = HALO_FLOATS * 4;
    const uint32_t bytes2 = (STAGE == 1 ? V_FLOATS : UN_FLOATS + V_FLOATS) * 4;
    int si = 0;
    // work: the strided items b, b + G, ... below full_items, then this CTA's tail segments
    // (item, first plane within the item, plane count), in increasing item order
    const int b = blockIdx.x;
    const int nfull = b < full_items ? (full_items - 1 - b) / (int)gridDim.x + 1 : 0;
    const int t0 = tail_begin[b], nwork = nfull + tail_begin[b + 1] - t0;

    for (int q = 0; q < nwork; ++q) {
        int gitem, k_off = 0, k_len = 1 << 30;
        if (q < nfull) {
            gitem = b + q * (int)gridDim.x;
        } else {
            const int4 sg = tail[t0 + q - nfull];
            gitem = sg.x;
            k_off = sg.y;
            k_len = sg.z;
        }
        while (si + 1 < nsolves && gitem >= D[si + 1].item_begin) ++si;
        const StageDesc &A = D[si];
        // the descriptor's scalars live in registers for the whole item (the mbarrier waits'
        // memory clobbers would otherwise reload them from global memory on every plane)
        const int nx = A.g.nx, nz = A.g.nz, nth = A.g.nth, pitch = A.g.pitch;
        const int64_t F = A.g.field, plane = A.g.plane;
        float *const out = A.out;
        const float2 dt2 = f2(A.dt, A.dt), cf2 = f2(A.coef, A.coef);
        // -velocity / (2 h) per axis turns weno3_2's 2 h u_x into the -V_d du/dx_d of L(u)
        const float hx2 = -0.5f * A.ihx, hz2 = -0.5f * A.ihz, ht2 = -0.5f * A.idth;
        float2 eps2[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) eps2[f] = f2(A.eps[f], A.eps[f]);
        const int item = gitem - A.item_begin;
        int xt = item % A.tiles_x;
        int rest = item / A.tiles_x;
        int zt = rest % A.tiles_z;
        int ch = rest / A.tiles_z;
        int k0 = ch * A.chunk + k_off;
        int kn = min(min(A.chunk, nth - ch * A.chunk) - k_off, k_len);
        int x0 = xt * TX, z0 = zt * TZ;
        int nplanes = kn + 4;
        auto plane_of = [&](int j) { return (k0 - 2 + j + 2 * nth) % nth; };
        auto issue = [&](int j) {
            int s = j % RING;
            mbar_expect_tx(bar + s, bytes_halo);
            tma_load_4d(ring + s * HALO_STRIDE, A.mapK, x0, z0, plane_of(j), 0, bar + s);
            pending |= 1u << s;
        };
        auto issue2 = [&](int j) {
            int s = j % RING2;
            mbar_expect_tx(bar2 + s, bytes2);
            float *dst = ring2 + s * SLOT2_STRIDE;
            int k = k0 + j;
            if (STAGE != 1) tma_load_4d(dst, A.mapN, x0 + XPAD, z0 + ZPAD, k, 0, bar2 + s);
            tma_load_4d(dst + UN_STRIDE, A.mapV, x0 + XPAD, z0 + ZPAD, k, 0, bar2 + s);
            pending2 |= 1u << s;
        };
        if (tid == 0) {
            for (int j = 0; j < min(RING, nplanes); ++j) issue(j);
            for (int j = 0; j < min(RING2, kn); ++j) issue2(j);
        }
        // A slot's parity flips and its pending bit clears only once its copy has been seen to
        // land: after a wait that gives up, the drain below still waits for that copy.
        const uint32_t polls = BOUNDED ? A.polls : DEFAULT_POLLS;
        bool ok = true;
        for (int j = 0; j < 4 && ok; ++j) {
            int s = j % RING;
            ok = mbar_wait_bounded(bar + s, (phase >> s) & 1u, polls);
            if (ok) {
                phase ^= 1u << s;
                if (tid == 0) pending &= ~(1u << s);
            }
        }
        const int iz = z0 + tz;
        const int ixa = x0 + 2 * tx;
        const bool row_ok = iz < nz;
        int sb = 0;  // kk % RING
        for (int kk = 0; kk < kn; ++kk, sb = (sb + 1 == RING ? 0 : sb + 1)) {
            {
                int s = sb + 4 >= RING ? sb + 4 - RING : sb + 4;
                if (ok) {
                    ok = mbar_wait_bounded(bar + s, (phase >> s) & 1u, polls);
                    if (ok) {
                        phase ^= 1u << s;
                        if (tid == 0) pending &= ~(1u << s);
                    }
                }
                int s2 = kk % RING2;
                if (ok) {
                    ok = mbar_wait_bounded(bar2 + s2, (phase2 >> s2) & 1u, polls);
                    if (ok) {
                        phase2 ^= 1u << s2;
                        if (tid == 0) pending2 &= ~(1u << s2);
                    }
                }
            }
            if (!ok) atomicOr(&abort_flag, 1);
            const int k = k0 + kk;
            const float *slot[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) slot[m] = ring + (sb + m >= RING ? sb + m - RING : sb + m) * HALO_STRIDE;
            const float *s2 = ring2 + (kk % RING2) * SLOT2_STRIDE;
            if (ok && row_ok && ixa < nx) {
                const int ci = (tz + 2) * HX + 2 * tx + 4;   // centre (first cell) in a halo slot
                const int cn = tz * TX + 2 * tx;             // centre in an interior slot
                const float2 vx = *reinterpret_cast<const float2 *>(s2 + UN_STRIDE + cn);
                const float2 vz = *reinterpret_cast<const float2 *>(s2 + UN_STRIDE + TZ * TX + cn);
                const float2 vt = *reinterpret_cast<const float2 *>(s2 + UN_STRIDE + 2 * TZ * TX + cn);
                const Up2 ux_up = upwind2(vx), uz_up = upwind2(vz), ut_up = upwind2(vt);
                const float2 cx = mul2(vx, f2(hx2, hx2)), cz = mul2(vz, f2(hz2, hz2)),
                             ct = mul2(vt, f2(ht2, ht2));
                float2 L[4];
                float2 ukc[NFIELD];
                auto gather = [&](int f, float2 sx[5], float2 sz[5], float2 st[5]) {
                    const float *c = slot[2] + f * HZ * HX + ci;
                    float2 a = *reinterpret_cast<const float2 *>(c - 2);
                    float2 b = *reinterpret_cast<const float2 *>(c);
                    float2 e = *reinterpret_cast<const float2 *>(c + 2);
                    sx[0] = a; sx[1] = f2(a.y, b.x); sx[2] = b; sx[3] = f2(b.y, e.x); sx[4] = e;
#pragma unroll
                    for (int m = 0; m < 5; ++m)
                        sz[m] = *reinterpret_cast<const float2 *>(c + (m - 2) * HX);
#pragma unroll
                    for (int m = 0; m < 5; ++m)
                        st[m] = *reinterpret_cast<const float2 *>(slot[m] + f * HZ * HX + ci);
                };
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    float2 sx[5], sz[5], st[5];
                    gather(f, sx, sz, st);
                    ukc[f] = sx[2];
                    // the angle label is continuous in x and z (no 2 pi seam inside a plane), so only
                    // its theta differences need wrapping
                    bool ang = (f == 2);
                    float2 ux = deriv2(sx, ux_up, eps2[f], false);
                    float2 uz = deriv2(sz, uz_up, eps2[f], false);
                    float2 ut = deriv2(st, ut_up, eps2[f], ang);
                    L[f] = fma2(cx, ux, fma2(cz, uz, mul2(ct, ut)));
                }
                {
                    float2 hx5[5], hz5[5], ht5[5], lx5[5], lz5[5], lt5[5];
                    gather(3, hx5, hz5, ht5);
                    gather(4, lx5, lz5, lt5);
                    ukc[3] = hx5[2];
                    ukc[4] = lx5[2];
                    float2 ux = deriv2_ff(hx5, lx5, ux_up, eps2[3]);
                    float2 uz = deriv2_ff(hz5, lz5, uz_up, eps2[3]);
                    float2 ut = deriv2_ff(ht5, lt5, ut_up, eps2[3]);
                    L[3] = add2(f2(1.f, 1.f), fma2(cx, ux, fma2(cz, uz, mul2(ct, ut))));
                }
                float2 un[NFIELD];
#pragma unroll
                for (int f = 0; f < NFIELD; ++f)
                    un[f] = (STAGE == 1) ? ukc[f] : *reinterpret_cast<const float2 *>(s2 + f * TZ * TX + cn);
                float2 o[NFIELD];
#pragma unroll
                for (int f = 0; f < 3; ++f)
                    o[f] = fma2(cf2, fma2(dt2, L[f], sub2(ukc[f], un[f])), un[f]);
                {
                    float2 inc = mul2(cf2, fma2(dt2, L[3], add2(sub2(ukc[3], un[3]), sub2(ukc[4], un[4]))));
                    ff ra = ff_add_f(un[3].x, un[4].x, inc.x);
                    ff rb = ff_add_f(un[3].y, un[4].y, inc.y);
                    o[3] = f2(ra.hi, rb.hi);
                    o[4] = f2(ra.lo, rb.lo);
                }
                // frozen cells of the source manifold carry a zeroed velocity copy
                const bool fa = vx.x == 0.f && vz.x == 0.f;
                const bool fb = vx.y == 0.f && vz.y == 0.f;
                const int64_t p = (int64_t)k * plane + (int64_t)(iz + ZPAD) * pitch + (ixa + XPAD);
#pragma unroll
                for (int f = 0; f < NFIELD; ++f) {
                    float2 v = f2(fa ? un[f].x : o[f].x, fb ? un[f].y : o[f].y);
                    if (ixa + 1 < nx) *reinterpret_cast<float2 *>(out + f * F + p) = v;
                    else out[f * F + p] = v.x;
                }
            }
            __syncthreads();
            if (abort_flag) break;
            if (tid == 0) {
                if (kk + RING < nplanes) issue(kk + RING);
                if (kk + RING2 < kn) issue2(kk + RING2);
            }
        }
        if (abort_flag) break;
    }
    if (abort_flag) {
        // latch the timeout and drain the copies this CTA still has in flight (with the default
        // bound: they were issued correctly and land, so the CTA never leaves with one pending)
        if (tid == 0) {
            atomicOr(err, DeviceErrors::TIMEOUT);
            for (int s = 0; s < RING; ++s)
                if (pending & (1u << s)) mbar_wait_bounded(bar + s, (phase >> s) & 1u);
            for (int s = 0; s < RING2; ++s)
                if (pending2 & (1u << s)) mbar_wait_bounded(bar2 + s, (phase2 >> s) & 1u);
        }
        __syncthreads();
    }
}

// ---- host side -----------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 4-D map over a padded field stack: dims {pitch, nz + 4, nth, nfields}, box {bx, bz, 1, nfields}.
static cudaError_t make_map(CUtensorMap *m, const Grid2D &g, float *base, int nfields, int bx, int bz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.nz + 2 * ZPAD), (cuuint64_t)g.nth,
                          (cuuint64_t)nfields};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.field * 4};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)bz, 1, (cuuint32_t)nfields};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

struct TmaMaps {
    CUtensorMap halo[3], inner[3], vel;  // host copies
    CUtensorMap *dev = nullptr;          // device copies: halo[0..2], inner[0..2], vel
    int chunk = 0;                       // theta-chunk length chosen by the autotuner
};

static const CUtensorMap *dmap_halo(const Solve &sv, int b) { return ((TmaMaps *)sv.tma)->dev + b; }
static const CUtensorMap *dmap_inner(const Solve &sv, int b) { return ((TmaMaps *)sv.tma)->dev + 3 + b; }
static const CUtensorMap *dmap_vel(const Solve &sv) { return ((TmaMaps *)sv.tma)->dev + 6; }

static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t tma_prepare(Solve &sv) {
    TmaMaps *m = new TmaMaps();
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
        e = make_map(&m->halo[b], sv.g, sv.state[b], NFIELD, tma::HX, tma::HZ);
        if (e == cudaSuccess) e = make_map(&m->inner[b], sv.g, sv.state[b], NFIELD, tma::TX, tma::TZ);
    }
    if (e == cudaSuccess) e = make_map(&m->vel, sv.g, sv.velp, 3, tma::TX, tma::TZ);
    if (e == cudaSuccess) e = cudaMalloc(&m->dev, 7 * sizeof(CUtensorMap));
    if (e == cudaSuccess) {
        CUtensorMap all[7] = {m->halo[0], m->halo[1], m->halo[2], m->inner[0], m->inner[1], m->inner[2], m->vel};
        e = cudaMemcpy(m->dev, all, sizeof all, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return e;
    }
    sv.tma = m;
    static bool attr_done = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_done) {
        cudaFuncSetAttribute(k_rk3_tma<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        cudaFuncSetAttribute(k_rk3_tma<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        cudaFuncSetAttribute(k_rk3_tma<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        cudaFuncSetAttribute(k_rk3_tma<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        cudaFuncSetAttribute(k_rk3_tma<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        cudaFuncSetAttribute(k_rk3_tma<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::SMEM_BYTES);
        attr_done = true;
    }
    return cudaGetLastError();
}

void tma_release(Solve &sv) {
    if (sv.tma) cudaFree(((TmaMaps *)sv.tma)->dev);
    delete (TmaMaps *)sv.tma;
    sv.tma = nullptr;
}

// Stage descriptor of solve `sv` for step r of a 3-step rotation starting at buffer cur0.
static StageDesc make_desc(const Solve &sv, int stage, int r, int chunk) {
    const Grid2D &g = sv.g;
    StageDesc A;
    A.g = g;
    A.dt = (float)sv.dt;
    A.ihx = (float)(1.0 / g.hx);
    A.ihz = (float)(1.0 / g.hz);
    A.idth = (float)(1.0 / g.dth);
    double h = g.hx > g.hz ? g.hx : g.hz;
    A.eps[0] = (float)(1e-6 * h * h);  // impact parameter (m)
    A.eps[1] = 1e-6f;                    // source indicator (dimensionless)
    A.eps[2] = (float)(1e-6 * g.dth * g.dth);
    A.eps[3] = (float)(1e-6 * (h / sv.c_ref) * (h / sv.c_ref));
    A.polls = sv.wait_polls ? sv.wait_polls : DEFAULT_POLLS;
    A.tiles_x = (g.nx + tma::TX - 1) / tma::TX;
    A.tiles_z = (g.nz + tma::TZ - 1) / tma::TZ;
    A.chunk = chunk > g.nth ? g.nth : chunk;
    A.items = A.tiles_x * A.tiles_z * ((g.nth + A.chunk - 1) / A.chunk);
    A.item_begin = 0;
    int n = (sv.cur + r) % 3, b1 = (n + 1) % 3, b2 = (n + 2) % 3;
    A.mapN = dmap_inner(sv, n);
    A.mapV = dmap_vel(sv);
    if (stage == 1) { A.mapK = dmap_halo(sv, n);  A.out = sv.state[b1]; A.coef = 1.f; }
    if (stage == 2) { A.mapK = dmap_halo(sv, b1); A.out = sv.state[b2]; A.coef = 0.25f; }
    if (stage == 3) { A.mapK = dmap_halo(sv, b2); A.out = sv.state[b1]; A.coef = 2.f / 3.f; }
    return A;
}

// Work split of a stage launch over its G = 2 x SMs CTAs.  The items (x tile, z tile, theta chunk)
// of the launch's solves, numbered in solve order, are strided over the CTAs (CTA b takes items
// b, b + G, ...) for the full rounds; the planes of the items of the last, partial round are cut
// into G contiguous runs of equal length, one per CTA.  (The 512^2 x 256 solve has 2752 items of
// 64 planes: nine rounds of 304 and 16 left over, which would otherwise run on 16 CTAs.  Measured:
// 0.5 % per stage launch; re-splitting the last two rounds instead was 0.5 % slower than plain
// striding.)  Launches with at most G items give each CTA one item.  Device layout: int4 segments [TAIL_SEGS_PER_CTA * G] (item, first
// plane in the item, planes, unused), then int begin[G + 1] (CTA b's segments are
// begin[b] .. begin[b + 1] - 1).
struct TailPlan {
    int grid = 0, full = 0;
    std::vector<int4> segs;
    std::vector<int> begin;
};

static int grid_ctas() { return sm_count() * tma::CTAS_PER_SM; }

size_t tail_plan_bytes() {
    size_t G = (size_t)grid_ctas();
    return tma::TAIL_SEGS_PER_CTA * G * sizeof(int4) + (G + 1) * sizeof(int);
}

// planes of item `gi` (a global item number) of the launch described by descs[0 .. n)
static int item_planes(const StageDesc *descs, int n, int gi) {
    int i = 0;
    while (i + 1 < n && gi >= descs[i + 1].item_begin) ++i;
    const StageDesc &d = descs[i];
    int ch = (gi - d.item_begin) / (d.tiles_x * d.tiles_z);
    int kn = d.g.nth - ch * d.chunk;
    return kn < d.chunk ? kn : d.chunk;
}

static TailPlan plan_tail(const StageDesc *descs, int n, int total) {
    TailPlan P;
    const int G = grid_ctas();
    P.begin.assign((size_t)G + 1, 0);
    P.grid = total < G ? total : G;
    P.full = total;
    if (total <= G) return P;
    P.full = (total / G) * G;
    if (P.full == total) return P;
    std::vector<int64_t> pre(1, 0);  // plane prefix over the remaining items
    for (int gi = P.full; gi < total; ++gi) pre.push_back(pre.back() + item_planes(descs, n, gi));
    const int64_t planes = pre.back();
    size_t it = 0;
    for (int cta = 0; cta < G; ++cta) {
        P.begin[cta] = (int)P.segs.size();
        int64_t lo = planes * cta / G, hi = planes * (cta + 1) / G;
        while (lo < hi) {
            while (pre[it + 1] <= lo) ++it;
            int64_t off = lo - pre[it], len = pre[it + 1] - lo;
            if (len > hi - lo) len = hi - lo;
            P.segs.push_back(make_int4(P.full + (int)it, (int)off, (int)len, 0));
            lo += len;
        }
    }
    P.begin[G] = (int)P.segs.size();
    if (P.segs.size() > (size_t)tma::TAIL_SEGS_PER_CTA * G) {  // cannot happen (< G items left); keep strides
        P.full = total;
        P.segs.clear();
        P.begin.assign((size_t)G + 1, 0);
    }
    return P;
}

static cudaError_t upload_tail(const TailPlan &P, void *d_tail, cudaStream_t s) {
    const int G = grid_ctas();
    char *base = (char *)d_tail;
    cudaError_t e = cudaSuccess;
    if (!P.segs.empty())
        e = cudaMemcpyAsync(base, P.segs.data(), P.segs.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + tma::TAIL_SEGS_PER_CTA * (size_t)G * sizeof(int4), P.begin.data(),
                            P.begin.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    return e;
}

static void launch_stage(int stage, const StageDesc *d, int nsolves, const TailPlan &P, void *d_tail,
                         unsigned *err, cudaStream_t s, bool bounded) {
    const int grid = P.grid;
    if (grid < 1) return;
    const int G = grid_ctas();
    const int4 *tail = (const int4 *)d_tail;
    const int *tb = (const int *)((const char *)d_tail + tma::TAIL_SEGS_PER_CTA * (size_t)G * sizeof(int4));
    const int T = tma::THREADS;
    const size_t M = tma::SMEM_BYTES;
    const int full = P.full;
    if (!bounded) {
        if (stage == 1) k_rk3_tma<1, false><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
        if (stage == 2) k_rk3_tma<2, false><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
        if (stage == 3) k_rk3_tma<3, false><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
    } else {
        if (stage == 1) k_rk3_tma<1, true><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
        if (stage == 2) k_rk3_tma<2, true><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
        if (stage == 3) k_rk3_tma<3, true><<<grid, T, M, s>>>(d, nsolves, full, tail, tb, err);
    }
}

int tma_chunk(const Solve &sv) { return sv.tma ? ((TmaMaps *)sv.tma)->chunk : 0; }

void tma_set_chunk(Solve &sv, int chunk) {
    if (sv.tma) ((TmaMaps *)sv.tma)->chunk = chunk;
}

// Autotuner: time stage 1 (reads u^n, writes a stage buffer, so the state is untouched) for each
// theta-chunk candidate and keep the fastest.  Synchronises the stream.
cudaError_t tma_autotune(Solve &sv, StageDesc *d_desc, void *d_tail, unsigned *err, cudaStream_t s) {
    static const int cand[4] = {8, 16, 32, 64};
    float best = 1e30f;
    int best_chunk = 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ci = 0; ci < 4; ++ci) {
        int ch = cand[ci];
        if (ch > sv.g.nth && ci > 0) break;
        StageDesc h = make_desc(sv, 1, 0, ch);
        cudaMemcpyAsync(d_desc, &h, sizeof h, cudaMemcpyHostToDevice, s);
        TailPlan P = plan_tail(&h, 1, h.items);
        cudaError_t eu = upload_tail(P, d_tail, s);
        if (eu != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return eu; }
        bool bounded = sv.wait_polls != 0;
        launch_stage(1, d_desc, 1, P, d_tail, err, s, bounded);  // warm
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; ++rep) launch_stage(1, d_desc, 1, P, d_tail, err, s, bounded);
        cudaEventRecord(e1, s);
        cudaError_t er = cudaEventSynchronize(e1);
        if (er != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return er; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_chunk = ch; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ((TmaMaps *)sv.tma)->chunk = best_chunk;
    return cudaGetLastError();
}

// Advance several FP32 solves together: per stage one persistent launch over the work items of all
// of them.  Whole 3-step rotations are captured once into a CUDA graph and replayed; the rest are
// launched directly.  After every step whose count (sv->steps, the steps before this call, plus the
// steps taken in it) is a multiple of BRANCH_SAMPLE, the solve's continued spreading argument is
// sampled.  d_desc must hold 9 * n descriptors; cap is a non-legacy stream for capture.
cudaError_t evolve_batch(Solve **sv, int n, int steps, StageDesc *d_desc, void *d_tail, unsigned *err,
                         cudaStream_t s, cudaStream_t cap) {
    if (n <= 0 || steps <= 0) return cudaSuccess;
    std::vector<StageDesc> h((size_t)9 * n);
    int total[9];
    for (int r = 0; r < 3; ++r)
        for (int st = 1; st <= 3; ++st) {
            int slot = r * 3 + (st - 1);
            int begin = 0;
            for (int i = 0; i < n; ++i) {
                StageDesc d = make_desc(*sv[i], st, r, tma_chunk(*sv[i]) ? tma_chunk(*sv[i]) : 16);
                d.item_begin = begin;
                begin += d.items;
                h[(size_t)slot * n + i] = d;
            }
            total[slot] = begin;
        }
    cudaError_t e = cudaMemcpyAsync(d_desc, h.data(), h.size() * sizeof(StageDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // the items (and so the work split) are the same for every stage and rotation phase
    const TailPlan P = plan_tail(h.data(), n, total[0]);
    e = upload_tail(P, d_tail, s);
    if (e != cudaSuccess) return e;
    bool bounded = false;  // any solve with a caller-set wait bound (they share their context's)
    for (int i = 0; i < n; ++i) bounded = bounded || sv[i]->wait_polls != 0;
    auto run_step = [&](int r, cudaStream_t st) {
        for (int stage = 1; stage <= 3; ++stage) {
            int slot = r * 3 + (stage - 1);
            launch_stage(stage, d_desc + (size_t)slot * n, n, P, d_tail, err, st, bounded);
        }
    };
    // step j of this call runs rotation phase j % 3; a rotation starting at a phase-0 step is one
    // launch of the captured graph (captured at its first use)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto rotation = [&]() -> cudaError_t {
        if (!exec) {
            cudaError_t er = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (er != cudaSuccess) return er;
            for (int r = 0; r < 3; ++r) run_step(r, cap);
            er = cudaStreamEndCapture(cap, &graph);
            if (er == cudaSuccess) er = cudaGraphInstantiate(&exec, graph, 0);
            if (er != cudaSuccess) return er;
        }
        return cudaGraphLaunch(exec, s);
    };
    int j = 0;
    while (j < steps && e == cudaSuccess) {
        // steps to the next branch sample of any solve (or to the end of the call)
        int seg = steps - j;
        for (int i = 0; i < n; ++i) {
            int to = BRANCH_SAMPLE - (int)((sv[i]->steps + j) % BRANCH_SAMPLE);
            seg = to < seg ? to : seg;
        }
        for (int q = j; q < j + seg && e == cudaSuccess;) {
            if (q % 3 == 0 && j + seg - q >= 3) {
                e = rotation();
                q += 3;
            } else {
                run_step(q % 3, s);
                ++q;
            }
        }
        j += seg;
        // one launch samples every due solve (per TRACK_BATCH solves)
        std::vector<Solve *> due;
        std::vector<const float *> due_st;
        for (int i = 0; i < n; ++i)
            if ((sv[i]->steps + j) % BRANCH_SAMPLE == 0) {
                due.push_back(sv[i]);
                due_st.push_back(sv[i]->state[(sv[i]->cur + j) % 3]);
            }
        if (e == cudaSuccess && !due.empty()) e = launch_track_batch(due.data(), due_st.data(), (int)due.size(), false, s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < n; ++i) sv[i]->cur = (sv[i]->cur + steps) % 3;
    return cudaGetLastError();
}

size_t stage_desc_bytes() { return sizeof(StageDesc); }

}  // namespace egb
