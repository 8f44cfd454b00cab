// Host side of the C ABI declared in include/cloth.h: handle lifetime,
// device memory, validation, CUDA-graph replay of substep blocks and error
// reporting.  No exception crosses the ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "cloth_internal.h"


namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(ClothHandle *h, cudaError_t e, const char *what)
{
    if (h) h->dead = true;
    return fail(CLOTH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CTRY(h, call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// Makes the handle's device current for the scope of one API call.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite3(const float *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

long long spring_count(long long nx, long long ny)
{
    long long s = nx * (ny - 1) + ny * (nx - 1) + 2 * (nx - 1) * (ny - 1);
    s += nx * (ny > 2 ? ny - 2 : 0) + ny * (nx > 2 ? nx - 2 : 0);
    return s;
}

const int kDR[CLOTH_NDIR] = {0, 1, 1, 1, 0, 2};
const int kDC[CLOTH_NDIR] = {1, 0, 1, -1, 2, 0};

void free_all(ClothHandle *h)
{
    for (cudaGraphExec_t &g : h->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    grid_free(&h->grid);
    cudaFree(h->state);
    cudaFree(h->pin_bits);
    cudaFree(h->ks_slot);
    cudaFree(h->kd_slot);
    cudaFree(h->ctrl);
    cudaFree(h->staging);
    cudaFree(h->coll_list);
    h->coll_list = nullptr;
    cudaFree(h->wind_tab);
    h->wind_tab = nullptr;
    cudaFree(h->force);
    h->force = nullptr;
    cudaFree(h->edge_resp);
    h->edge_resp = nullptr;
    cudaFree(h->edge_hit);
    h->edge_hit = nullptr;
    cudaFree(h->edge_stamp);
    h->edge_stamp = nullptr;
    cudaFree(h->edge_more);
    h->edge_more = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->state = nullptr;
    h->pin_bits = nullptr;
    h->ks_slot = h->kd_slot = nullptr;
    h->ctrl = nullptr;
    h->staging = nullptr;
    h->cap_stream = nullptr;
}

}  // namespace

// Derives the kernel parameters from the handle's description and buffers.
// The fractional part of x (turns) as a 64-bit binary fraction of a turn.
static unsigned long long turn_fraction(double x)
{
    const double f = x - floor(x);  // [0, 1)
    const double scaled = f * 18446744073709551616.0;  // 2^64
    return scaled >= 18446744073709551616.0 ? 0ull : (unsigned long long)scaled;
}

void cloth_fill_params(ClothHandle *h)
{
    const ClothDesc &d = h->desc;
    StepParams &p = h->params;
    h->params_gen++;
    p.nx = d.nx;
    p.ny = d.ny;
    p.n = h->n;
    p.pitch = h->pitch;
    p.rows_per_warp = substep_rows_per_warp(d.nx, d.ny, h->sm_count);
    substep_shape(p);
    p.stride = h->stride;
    p.parity = -1;
    p.state0 = h->state;
    p.state1 = h->state + 6 * h->stride;
    p.pin_bits = h->pin_bits;
    p.ks_slot = h->ks_slot;
    p.kd_slot = h->kd_slot;
    for (int a = 0; a < 3; a++) {
        p.ks[a] = d.ks[a];
        p.kd[a] = d.kd[a];
        p.g[a] = d.gravity[a];
        p.pin_vel[a] = d.pin_velocity[a];
        p.w_dir[a] = d.wind.dir[a];
    }
    // rest lengths of the six directions from the flat grid, in double
    for (int k = 0; k < CLOTH_NDIR; k++) {
        double l2 = 0.0;
        for (int a = 0; a < 3; a++) {
            const double e = (double)kDC[k] * d.du[a] + (double)kDR[k] * d.dv[a];
            l2 += e * e;
        }
        p.L0[k] = (float)sqrt(l2);
    }
    const double dt_s = (double)d.dt / (double)d.substeps;
    p.dt = (float)dt_s;
    p.inv_mass = (float)((double)h->n / (double)d.total_mass);
    p.has_wind = d.wind.amp != 0.0f;
    p.w_amp = d.wind.amp;
    const double two_pi = 6.283185307179586;
    p.w_turn_step = turn_fraction((double)d.wind.freq * dt_s);  // omega / 2 pi, turns per substep
    double k0 = 0.0, kc = 0.0, kr = 0.0;
    for (int a = 0; a < 3; a++) {
        k0 += (double)d.wind.udir[a] * d.origin[a];
        kc += (double)d.wind.udir[a] * d.du[a];
        kr += (double)d.wind.udir[a] * d.dv[a];
    }
    p.w_turn0 = turn_fraction(((double)d.wind.phase + (double)d.wind.kappa * k0) / two_pi);
    p.w_kc = (float)((double)d.wind.kappa * kc);
    p.w_kr = (float)((double)d.wind.kappa * kr);
    p.wind_rows = h->wind_tab;
    p.wind_cols = h->wind_tab ? h->wind_tab + d.ny : nullptr;
    p.has_mesh = h->has_mesh;
    p.tri = h->grid.tri;
    p.cell_start = h->grid.cell_start;
    p.tri_ids = h->grid.tri_ids;
    p.etri = h->grid.etri;
    for (int a = 0; a < 3; a++) {
        p.go[a] = h->grid.origin[a];
        p.gd[a] = h->grid.dims[a];
    }
    p.ginv = h->grid.inv;
    // nodes whose path box reaches the box of the mesh's vertices are listed for
    // the narrow phase (a path outside it meets no triangle); the box is padded
    // by 1e-4 of its largest side, far above float32 rounding of the test
    double ext = 0.0;
    for (int a = 0; a < 3; a++)
        if (h->has_mesh) ext = fmax(ext, (double)h->grid.hi[a] - (double)h->grid.lo[a]);
    const double pad = 1e-4 * ext + 1e-6;
    for (int a = 0; a < 3; a++) {
        p.mlo[a] = h->has_mesh ? (float)((double)h->grid.lo[a] - pad) : 0.0f;
        p.mhi[a] = h->has_mesh ? (float)((double)h->grid.hi[a] + pad) : 0.0f;
    }
    p.delta = d.contact_offset;
    p.eps = d.mt_eps;
    p.tmin = d.mt_t_min;
    p.restitution = d.restitution;
    p.ctrl = h->ctrl;
    p.force = h->force;
    p.edge_resp = h->edge_resp;
    p.edge_hit = h->edge_hit;
    p.edge_stamp = h->edge_stamp;
    p.edge_more = h->edge_more;
    p.coll_list = h->coll_list;
    p.coll_count = h->ctrl ? &h->ctrl->coll_count : nullptr;
    p.coll_blocks = h->sm_count * CLOTH_COLL_CTAS_PER_SM;
}

namespace {

void invalidate_graph(ClothHandle *h)
{
    for (cudaGraphExec_t &g : h->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// One substep launched with its buffer parity (k & 1 of that substep).
cudaError_t launch_substep_parity(const ClothHandle *h, long long k, cudaStream_t s)
{
    StepParams q = h->params;
    q.parity = (int)(k & 1);
    return launch_substep(q, s);
}

// Capture one step (desc.substeps launches) whose first substep has parity
// par as a graph on a private stream.
cudaError_t ensure_graph(ClothHandle *h, int par)
{
    if (h->graph[par]) return cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < h->desc.substeps && le == cudaSuccess; s++) le = launch_substep_parity(h, par + s, h->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&h->graph[par], g, 0);
    cudaGraphDestroy(g);
    return e;
}

int check_handle(ClothHandle *h)
{
    if (!h) return fail(CLOTH_ERR_INVALID_ARG, "null handle");
    if (h->dead) return fail(CLOTH_ERR_STATE, "handle unusable after an earlier CUDA error");
    return CLOTH_OK;
}

int read_flags(ClothHandle *h, unsigned *flags)
{
    CTRY(h, cudaMemcpyAsync(flags, &h->ctrl->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream),
         "read device flags");
    CTRY(h, cudaStreamSynchronize(h->stream), "synchronize");
    return CLOTH_OK;
}

int flags_status(unsigned flags)
{
    if (flags & CTRL_FLAG_TIMEOUT) return fail(CLOTH_ERR_TIMEOUT, "a device-side wait timed out");
    if (flags & CTRL_FLAG_NONFINITE) return fail(CLOTH_ERR_NONFINITE, "state became non-finite");
    if (flags & CTRL_FLAG_PARITY) return fail(CLOTH_ERR_STATE, "a substep ran on the wrong state buffer (internal)");
    return CLOTH_OK;
}

// Host array -> device buffer (synchronous for pageable memory).
cudaError_t upload(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

}  // namespace

// Lets other translation units report through cloth_last_error().
void cloth_set_error_message(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

extern "C" {

const char *cloth_last_error(void) { return g_err; }

int cloth_create(const ClothDesc *desc, void *stream, ClothHandle **out)
{
    if (!out) return fail(CLOTH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(CLOTH_ERR_INVALID_ARG, "desc is NULL");
    const ClothDesc &d = *desc;
    if (d.nx < 1 || d.ny < 1) return fail(CLOTH_ERR_INVALID_ARG, "nx, ny must be >= 1");
    const long long N = (long long)d.nx * d.ny;
    if (N > (1ll << 30)) return fail(CLOTH_ERR_INVALID_ARG, "too many nodes (%lld)", N);
    // kernels index a plane with 32-bit offsets r * pitch + c
    if ((long long)((d.nx + 3) / 4 * 4) * d.ny >= (1ll << 31))
        return fail(CLOTH_ERR_INVALID_ARG, "plane of %d x %d nodes too large", d.nx, d.ny);
    // and the six planes of a state buffer with 32-bit offsets j * stride + o
    if (6 * (((long long)((d.nx + 3) / 4 * 4) * d.ny + 63) / 64 * 64) >= (1ll << 32))
        return fail(CLOTH_ERR_INVALID_ARG, "plane of %d x %d nodes too large for 32-bit state offsets", d.nx, d.ny);
    if (d.substeps < 1) return fail(CLOTH_ERR_INVALID_ARG, "substeps must be >= 1");
    if (!(d.dt > 0.0f) || !isfinite(d.dt)) return fail(CLOTH_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!(d.total_mass > 0.0f) || !isfinite(d.total_mass))
        return fail(CLOTH_ERR_INVALID_ARG, "total_mass must be finite and > 0");
    if (!finite3(d.origin) || !finite3(d.du) || !finite3(d.dv) || !finite3(d.ks) || !finite3(d.kd) ||
        !finite3(d.gravity) || !finite3(d.wind.dir) || !finite3(d.wind.udir) || !isfinite(d.wind.amp) ||
        !isfinite(d.wind.freq) || !isfinite(d.wind.kappa) || !isfinite(d.wind.phase) || !isfinite(d.contact_offset) ||
        !isfinite(d.mt_eps) || !isfinite(d.mt_t_min) || !isfinite(d.restitution) || !finite3(d.pin_velocity))
        return fail(CLOTH_ERR_INVALID_ARG, "non-finite parameter in desc");
    const long long S = spring_count(d.nx, d.ny);
    if (d.init_pos)
        for (long long i = 0; i < 3 * N; i++)
            if (!isfinite(d.init_pos[i])) return fail(CLOTH_ERR_INVALID_ARG, "non-finite init_pos[%lld]", i);
    if (d.init_vel)
        for (long long i = 0; i < 3 * N; i++)
            if (!isfinite(d.init_vel[i])) return fail(CLOTH_ERR_INVALID_ARG, "non-finite init_vel[%lld]", i);
    if (d.ks_spring)
        for (long long i = 0; i < S; i++)
            if (!isfinite(d.ks_spring[i])) return fail(CLOTH_ERR_INVALID_ARG, "non-finite ks_spring[%lld]", i);
    if (d.kd_spring)
        for (long long i = 0; i < S; i++)
            if (!isfinite(d.kd_spring[i])) return fail(CLOTH_ERR_INVALID_ARG, "non-finite kd_spring[%lld]", i);

    ClothHandle *h = new (std::nothrow) ClothHandle();
    if (!h) return fail(CLOTH_ERR_OOM, "host allocation failed");
    h->desc = d;
    h->desc.ks_spring = h->desc.kd_spring = nullptr;
    h->desc.init_pos = h->desc.init_vel = nullptr;
    h->desc.pinned = nullptr;
    h->n = (int)N;
    h->pitch = (d.nx + 3) / 4 * 4;                                          // 16-byte aligned rows
    h->stride = ((long long)h->pitch * d.ny + 63) / 64 * 64;                // 256-byte aligned planes
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        h->sm_count < 1)
        h->sm_count = 152;
    cudaGetLastError();

    int rc = CLOTH_OK;
    cudaError_t e = cudaSuccess;
    try {
    do {
        if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaMalloc(&h->state, sizeof(float) * 12 * (size_t)h->stride)) != cudaSuccess) break;
        if ((e = cudaMalloc(&h->ctrl, sizeof(DevCtrl))) != cudaSuccess) break;
        if ((e = cudaMalloc(&h->staging, sizeof(float) * 6 * (size_t)N)) != cudaSuccess) break;
        if ((e = cudaMalloc(&h->coll_list, sizeof(int) * (size_t)N)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(h->ctrl, 0, sizeof(DevCtrl), h->stream)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(h->state, 0, sizeof(float) * 12 * (size_t)h->stride, h->stream)) != cudaSuccess)
            break;
        // initial state: given arrays, else the flat grid (computed in double) at rest
        std::vector<float> init(6 * (size_t)N, 0.0f);
        for (long long i = 0; i < N; i++) {
            const long long r = i / d.nx, c = i % d.nx;
            for (int a = 0; a < 3; a++) {
                init[3 * i + a] = d.init_pos ? d.init_pos[3 * i + a]
                                             : (float)((double)d.origin[a] + (double)c * d.du[a] + (double)r * d.dv[a]);
                init[3 * N + 3 * i + a] = d.init_vel ? d.init_vel[3 * i + a] : 0.0f;
            }
        }
        if ((e = upload(h->staging, init.data(), sizeof(float) * 6 * (size_t)N, h->stream)) != cudaSuccess) break;
        if ((e = launch_aos_to_soa(h->staging, h->staging + 3 * N, h->state, h->state + 6 * h->stride, h->stride,
                                   (int)N, d.nx, h->pitch, h->ctrl, h->stream)) != cudaSuccess)
            break;
        if (d.pinned) {
            // one bit per padded position r*pitch + c
            const long long nb = (long long)h->pitch * d.ny;
            std::vector<uint32_t> bits((size_t)(nb + 31) / 32, 0u);
            bool any = false;
            for (long long i = 0; i < N; i++)
                if (d.pinned[i]) {
                    const long long b = (i / d.nx) * h->pitch + (i % d.nx);
                    bits[(size_t)(b >> 5)] |= 1u << (b & 31);
                    any = true;
                }
            if (any) {
                if ((e = cudaMalloc(&h->pin_bits, sizeof(uint32_t) * bits.size())) != cudaSuccess) break;
                if ((e = upload(h->pin_bits, bits.data(), sizeof(uint32_t) * bits.size(), h->stream)) != cudaSuccess)
                    break;
            }
        }
        if (d.flags & CLOTH_FLAG_EDGE_COLLISION) {
            if ((e = cudaMalloc(&h->edge_resp, sizeof(float4) * (size_t)N)) != cudaSuccess) break;
            if ((e = cudaMalloc(&h->edge_hit, sizeof(float4) * 3 * (size_t)h->stride)) != cudaSuccess) break;
            if ((e = cudaMalloc(&h->edge_more, sizeof(float4) * CLOTH_EDGE_MORE * 3 * (size_t)h->stride)) !=
                cudaSuccess)
                break;
            if ((e = cudaMalloc(&h->edge_stamp, sizeof(unsigned long long) * (size_t)h->stride)) != cudaSuccess) break;
            if ((e = cudaMemsetAsync(h->edge_stamp, 0, sizeof(unsigned long long) * (size_t)h->stride, h->stream)) != cudaSuccess)
                break;
        }
        if (d.flags & CLOTH_FLAG_ATOMIC_SPRINGS) {
            const size_t nf = (size_t)h->pitch * d.ny;
            if ((e = cudaMalloc(&h->force, sizeof(float4) * nf)) != cudaSuccess) break;
            if ((e = cudaMemsetAsync(h->force, 0, sizeof(float4) * nf, h->stream)) != cudaSuccess) break;
        }
        if (d.wind.amp != 0.0f) {
            // (sin, cos) of kappa*(udir.dv)*row and kappa*(udir.du)*col, in double
            double kc = 0.0, kr = 0.0;
            for (int a = 0; a < 3; a++) {
                kc += (double)d.wind.udir[a] * d.du[a];
                kr += (double)d.wind.udir[a] * d.dv[a];
            }
            kc *= d.wind.kappa;
            kr *= d.wind.kappa;
            std::vector<float2> tab((size_t)d.ny + d.nx);
            for (long long r = 0; r < d.ny; r++) tab[r] = make_float2((float)sin(kr * r), (float)cos(kr * r));
            for (long long c = 0; c < d.nx; c++)
                tab[d.ny + c] = make_float2((float)sin(kc * c), (float)cos(kc * c));
            if ((e = cudaMalloc(&h->wind_tab, sizeof(float2) * tab.size())) != cudaSuccess) break;
            if ((e = upload(h->wind_tab, tab.data(), sizeof(float2) * tab.size(), h->stream)) != cudaSuccess) break;
        }
        if (d.ks_spring || d.kd_spring) {
            // canonical order -> [direction][owner node] slots
            std::vector<float> ks(6 * (size_t)h->stride, 0.0f), kd(6 * (size_t)h->stride, 0.0f);
            const int type[CLOTH_NDIR] = {0, 0, 1, 1, 2, 2};
            long long s = 0;
            for (long long r = 0; r < d.ny; r++)
                for (long long c = 0; c < d.nx; c++)
                    for (int k = 0; k < CLOTH_NDIR; k++) {
                        const long long r2 = r + kDR[k], c2 = c + kDC[k];
                        if (r2 < 0 || r2 >= d.ny || c2 < 0 || c2 >= d.nx) continue;
                        const size_t slot = (size_t)k * h->stride + (size_t)(r * h->pitch + c);
                        ks[slot] = d.ks_spring ? d.ks_spring[s] : d.ks[type[k]];
                        kd[slot] = d.kd_spring ? d.kd_spring[s] : d.kd[type[k]];
                        s++;
                    }
            if ((e = cudaMalloc(&h->ks_slot, sizeof(float) * ks.size())) != cudaSuccess) break;
            if ((e = cudaMalloc(&h->kd_slot, sizeof(float) * kd.size())) != cudaSuccess) break;
            if ((e = upload(h->ks_slot, ks.data(), sizeof(float) * ks.size(), h->stream)) != cudaSuccess) break;
            if ((e = upload(h->kd_slot, kd.data(), sizeof(float) * kd.size(), h->stream)) != cudaSuccess) break;
        }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) break;
    } while (0);
    } catch (...) {
        cudaStreamSynchronize(h->stream);
        free_all(h);
        delete h;
        return fail(CLOTH_ERR_OOM, "host allocation failed");
    }
    if (e != cudaSuccess) {
        rc = (e == cudaErrorMemoryAllocation) ? fail(CLOTH_ERR_OOM, "device allocation failed: %s", cudaGetErrorString(e))
                                              : cuda_fail(nullptr, e, "cloth_create");
        free_all(h);
        delete h;
        cudaGetLastError();
        return rc;
    }
    cloth_fill_params(h);
    *out = h;
    return CLOTH_OK;
}

int cloth_set_mesh(ClothHandle *h, const float *verts, int32_t nverts, const int32_t *tris, int32_t ntris)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (ntris < 0 || nverts < 0) return fail(CLOTH_ERR_BAD_MESH, "negative mesh size");
    if (ntris > 0 && (!verts || !tris || nverts < 1)) return fail(CLOTH_ERR_BAD_MESH, "missing mesh arrays");
    for (long long i = 0; i < 3 * (long long)ntris; i++)
        if (tris[i] < 0 || tris[i] >= nverts)
            return fail(CLOTH_ERR_BAD_MESH, "triangle index %d at %lld out of range [0, %d)", tris[i], i, nverts);
    for (long long i = 0; i < 3 * (long long)nverts && ntris > 0; i++)
        if (!isfinite(verts[i])) return fail(CLOTH_ERR_BAD_MESH, "non-finite vertex coordinate at %lld", i);
    DeviceScope ds(h->device);
    CTRY(h, cudaStreamSynchronize(h->stream), "synchronize");
    DevGrid g{};
    if (ntris > 0) {
        if (grid_params(verts, tris, ntris, &g.h, g.origin, g.dims, &g.inv) != 0)
            return fail(CLOTH_ERR_BAD_MESH, "grid parameters");
        for (int a = 0; a < 3; a++) {
            g.lo[a] = INFINITY;
            g.hi[a] = -INFINITY;
        }
        for (long long i = 0; i < 3 * (long long)ntris; i++)
            for (int a = 0; a < 3; a++) {
                const float x = verts[3 * (long long)tris[i] + a];
                g.lo[a] = fminf(g.lo[a], x);
                g.hi[a] = fmaxf(g.hi[a], x);
            }
        float *dv = nullptr;
        int *dt = nullptr;
        cudaError_t e = cudaMalloc(&dv, sizeof(float) * 3 * (size_t)nverts);
        if (e == cudaSuccess) e = cudaMalloc(&dt, sizeof(int) * 3 * (size_t)ntris);
        if (e == cudaSuccess) e = upload(dv, verts, sizeof(float) * 3 * (size_t)nverts, h->stream);
        if (e == cudaSuccess) e = upload(dt, tris, sizeof(int) * 3 * (size_t)ntris, h->stream);
        if (e == cudaSuccess) e = grid_build(dv, dt, ntris, &g, h->stream);
        cudaFree(dv);
        cudaFree(dt);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            return fail(CLOTH_ERR_BAD_MESH, "mesh needs more than 2^31 grid entries");
        }
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(CLOTH_ERR_OOM, "device allocation failed while building the grid");
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "grid build");
    }
    grid_free(&h->grid);
    h->grid = g;
    h->has_mesh = ntris > 0;
    cloth_fill_params(h);
    invalidate_graph(h);
    return CLOTH_OK;
}

int cloth_step(ClothHandle *h, int32_t nsteps)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(CLOTH_ERR_INVALID_ARG, "nsteps < 0");
    if (nsteps == 0) return CLOTH_OK;
    DeviceScope ds(h->device);
    // substeps_done is the device's substep counter k as of this call's first
    // launch (every path that queues substeps adds them), so each launch knows
    // its buffer parity
    const long long S = h->desc.substeps;
    if (h->desc.flags & CLOTH_FLAG_NO_GRAPH) {
        for (long long j = 0; j < (long long)nsteps * S; j++)
            CTRY(h, launch_substep_parity(h, h->substeps_done + j, h->stream), "substep launch");
    } else {
        for (long long s = 0; s < nsteps; s++) {
            const int par = (int)((h->substeps_done + s * S) & 1);
            CTRY(h, ensure_graph(h, par), "graph capture");
            CTRY(h, cudaGraphLaunch(h->graph[par], h->stream), "graph launch");
        }
    }
    h->substeps_done += (long long)nsteps * h->desc.substeps;
    return CLOTH_OK;
}

int cloth_read(ClothHandle *h, float *pos_out, float *vel_out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceScope ds(h->device);
    const long long N = h->n;
    unsigned flags = 0;
    if (pos_out || vel_out) {
        CTRY(h, launch_soa_to_aos(h->state, h->state + 6 * h->stride, h->stride, h->n, h->desc.nx, h->pitch, h->ctrl,
                                  pos_out ? h->staging : nullptr, vel_out ? h->staging + 3 * N : nullptr, h->stream),
             "state gather");
        if (pos_out)
            CTRY(h, cudaMemcpyAsync(pos_out, h->staging, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->stream),
                 "copy positions");
        if (vel_out)
            CTRY(h, cudaMemcpyAsync(vel_out, h->staging + 3 * N, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost,
                                    h->stream),
                 "copy velocities");
    }
    rc = read_flags(h, &flags);
    if (rc) return rc;
    return flags_status(flags);
}

int cloth_set_state(ClothHandle *h, const float *pos, const float *vel)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!pos && !vel) return CLOTH_OK;
    DeviceScope ds(h->device);
    const long long N = h->n;
    if (pos) CTRY(h, upload(h->staging, pos, sizeof(float) * 3 * N, h->stream), "upload positions");
    if (vel) CTRY(h, upload(h->staging + 3 * N, vel, sizeof(float) * 3 * N, h->stream), "upload velocities");
    CTRY(h, launch_aos_to_soa(pos ? h->staging : nullptr, vel ? h->staging + 3 * N : nullptr, h->state,
                              h->state + 6 * h->stride, h->stride, h->n, h->desc.nx, h->pitch, h->ctrl, h->stream),
         "state scatter");
    return CLOTH_OK;
}

int cloth_compute_normals(ClothHandle *h, float *d_normals)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!d_normals) return fail(CLOTH_ERR_INVALID_ARG, "d_normals is NULL");
    DeviceScope ds(h->device);
    // the current state buffer: substeps_done counts every substep queued so far
    const float *cur = h->state + ((h->substeps_done & 1) ? 6 * h->stride : 0);
    CTRY(h, launch_normals(cur, h->stride, h->desc.nx, h->desc.ny, h->pitch, d_normals, h->sm_count, h->stream),
         "normals");
    return CLOTH_OK;
}

int cloth_profile_substeps(ClothHandle *h, int32_t nsub, float *walk_us, float *collide_us)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (nsub < 1 || nsub > 4096) return fail(CLOTH_ERR_INVALID_ARG, "nsub must be in [1, 4096]");
    DeviceScope ds(h->device);
    const int ne = 3 * nsub;
    std::vector<cudaEvent_t> ev(ne, nullptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < ne && e == cudaSuccess; i++) e = cudaEventCreate(&ev[i]);
    // captured into a graph, so the GPU runs the launches back to back
    // instead of waiting for the host between them
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        // external records: timestamp nodes in the graph, not capture-internal joins
        auto rec = [&](cudaEvent_t x) { return cudaEventRecordWithFlags(x, h->cap_stream, cudaEventRecordExternal); };
        for (int i = 0; i < nsub && le == cudaSuccess; i++) {
            le = rec(ev[3 * i]);
            if (le == cudaSuccess) le = launch_walk(h->params, h->cap_stream);
            if (le == cudaSuccess) le = rec(ev[3 * i + 1]);
            if (le == cudaSuccess && h->has_mesh) le = launch_collide(h->params, h->cap_stream);
            if (le == cudaSuccess) le = rec(ev[3 * i + 2]);
        }
        e = cudaStreamEndCapture(h->cap_stream, &g);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    double tw = 0.0, tc = 0.0;
    for (int i = 0; i < nsub && e == cudaSuccess; i++) {
        float a = 0.0f, b = 0.0f;
        e = cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]);
        tw += a;
        tc += b;
    }
    for (int i = 0; i < ne; i++)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(h, e, "profiled substeps");
    h->substeps_done += nsub;
    if (walk_us) *walk_us = (float)(1e3 * tw / nsub);
    if (collide_us) *collide_us = h->has_mesh ? (float)(1e3 * tc / nsub) : 0.0f;
    unsigned flags = 0;
    rc = read_flags(h, &flags);
    if (rc) return rc;
    return flags_status(flags);
}

int cloth_sync(ClothHandle *h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceScope ds(h->device);
    unsigned flags = 0;
    rc = read_flags(h, &flags);
    if (rc) return rc;
    return flags_status(flags);
}

int cloth_get_collision_stats(ClothHandle *h, int64_t *listed, int64_t *tested, int64_t *hits)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceScope ds(h->device);
    unsigned long long v[3] = {0ull, 0ull, 0ull};
    CTRY(h, cudaMemcpyAsync(v, &h->ctrl->stat_listed, sizeof(v), cudaMemcpyDeviceToHost, h->stream),
         "read collision statistics");
    CTRY(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (listed) *listed = (int64_t)v[0];
    if (tested) *tested = (int64_t)v[1];
    if (hits) *hits = (int64_t)v[2];
    return CLOTH_OK;
}

void cloth_destroy(ClothHandle *h)
{
    if (!h) return;
    {
        DeviceScope ds(h->device);
        cudaStreamSynchronize(h->stream);
        free_all(h);
        cudaGetLastError();
    }
    delete h;
}

int cloth_get_info(ClothHandle *h, ClothInfo *info)
{
    if (!h || !info) return fail(CLOTH_ERR_INVALID_ARG, "null argument");
    memset(info, 0, sizeof(*info));
    info->nx = h->desc.nx;
    info->ny = h->desc.ny;
    info->n = h->n;
    info->substeps = h->desc.substeps;
    info->substeps_done = h->substeps_done;
    info->plane_stride = h->stride;
    float *cur = h->state + ((h->substeps_done & 1) ? 6 * h->stride : 0);
    for (int a = 0; a < 3; a++) {
        info->pos_planes[a] = cur + a * h->stride;
        info->vel_planes[a] = cur + (3 + a) * h->stride;
        info->grid_dims[a] = h->has_mesh ? h->grid.dims[a] : 0;
        info->grid_origin[a] = h->has_mesh ? h->grid.origin[a] : 0.0f;
    }
    info->ntris = h->has_mesh ? h->grid.ntris : 0;
    info->grid_h = h->has_mesh ? h->grid.h : 0.0f;
    info->grid_inv = h->has_mesh ? h->grid.inv : 0.0f;
    info->grid_entries = h->has_mesh ? h->grid.nentries : 0;
    info->has_per_spring = h->ks_slot != nullptr;
    info->row_pitch = h->pitch;
    return h->dead ? fail(CLOTH_ERR_STATE, "handle unusable after an earlier CUDA error") : CLOTH_OK;
}

int cloth_get_grid(ClothHandle *h, int32_t *cell_start, int32_t *tri_ids)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->has_mesh) return fail(CLOTH_ERR_INVALID_ARG, "no mesh set");
    DeviceScope ds(h->device);
    if (cell_start)
        CTRY(h, cudaMemcpyAsync(cell_start, h->grid.cell_start, sizeof(int) * (size_t)(h->grid.ncells + 1),
                                cudaMemcpyDeviceToHost, h->stream),
             "copy cell_start");
    if (tri_ids && h->grid.nentries > 0)
        CTRY(h, cudaMemcpyAsync(tri_ids, h->grid.tri_ids, sizeof(int) * (size_t)h->grid.nentries,
                                cudaMemcpyDeviceToHost, h->stream),
             "copy tri_ids");
    CTRY(h, cudaStreamSynchronize(h->stream), "synchronize");
    return CLOTH_OK;
}

int cloth_query_candidates(ClothHandle *h, const float *S, const float *E, int32_t nseg, int32_t *counts,
                           int32_t *ids, int32_t cap)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (nseg < 0 || cap < 0 || (nseg > 0 && (!S || !E || !counts)) || (cap > 0 && !ids))
        return fail(CLOTH_ERR_INVALID_ARG, "bad query arguments");
    if (!h->has_mesh) return fail(CLOTH_ERR_INVALID_ARG, "no mesh set");
    if (nseg == 0) return CLOTH_OK;
    DeviceScope ds(h->device);
    float *dS = nullptr, *dE = nullptr;
    int *dc = nullptr, *di = nullptr;
    const size_t nb = sizeof(float) * 3 * (size_t)nseg;
    const size_t ib = sizeof(int) * (size_t)nseg * (size_t)(cap > 0 ? cap : 1);
    cudaError_t e = cudaMalloc(&dS, nb);
    if (e == cudaSuccess) e = cudaMalloc(&dE, nb);
    if (e == cudaSuccess) e = cudaMalloc(&dc, sizeof(int) * (size_t)nseg);
    if (e == cudaSuccess) e = cudaMalloc(&di, ib);
    if (e == cudaSuccess) e = upload(dS, S, nb, h->stream);
    if (e == cudaSuccess) e = upload(dE, E, nb, h->stream);
    if (e == cudaSuccess) e = grid_query(h->grid, dS, dE, nseg, dc, di, cap, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, dc, sizeof(int) * (size_t)nseg, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && cap > 0) e = cudaMemcpyAsync(ids, di, ib, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dS);
    cudaFree(dE);
    cudaFree(dc);
    cudaFree(di);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(CLOTH_ERR_OOM, "device allocation failed");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "candidate query");
    return CLOTH_OK;
}

}  // extern "C"
