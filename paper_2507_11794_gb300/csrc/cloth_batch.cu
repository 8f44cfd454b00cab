// Host side of the batch API: many independent cloths (each with its own
// grid, constants and surface model) advanced together by one persistent walk
// launch and one collision launch per substep, replayed from a CUDA graph.
// Not in the paper, which steps one cloth per frame; the batch keeps every
// cloth's arithmetic identical to stepping it alone.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cloth_internal.h"

struct ClothBatch {
    std::vector<ClothHandle *> cl;
    int device = 0;
    int sm_count = 152;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    DevCtrl *ctrl = nullptr;
    unsigned *work = nullptr;
    int *coll_list = nullptr;
    int *coll_cloth = nullptr;
    StepParams *d_params = nullptr;
    int4 *d_items = nullptr;
    int n_items = 0;
    int rows_per_warp = 8;
    int ctas_per_sm = 2;
    int substeps = 1;
    BatchArgs args{};
    cudaGraphExec_t graph = nullptr;
    long long substeps_done = 0;
    bool dead = false;
};

namespace {

int bfail(int code, const char *fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    cloth_set_error_message(msg);
    return code;
}

int bcuda(ClothBatch *b, cudaError_t e, const char *what)
{
    if (b) b->dead = true;
    return bfail(CLOTH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define BTRY(b, call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

int check_batch(ClothBatch *b)
{
    if (!b) return bfail(CLOTH_ERR_INVALID_ARG, "null batch");
    if (b->dead) return bfail(CLOTH_ERR_STATE, "batch unusable after an earlier CUDA error");
    return CLOTH_OK;
}

// Parameters of every cloth for the current tuning, and the item list sorted
// longest first (ties: cloth, strip row, strip column).
cudaError_t rebuild(ClothBatch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    const int scols = substep_strip_cols();
    std::vector<StepParams> prm(b->cl.size());
    std::vector<int4> items;
    for (size_t i = 0; i < b->cl.size(); i++) {
        ClothHandle *h = b->cl[i];
        cloth_fill_params(h);
        StepParams p = h->params;
        p.rows_per_warp = b->rows_per_warp;
        substep_shape(p);
        p.ctrl = b->ctrl;
        p.coll_list = b->coll_list;
        p.coll_cloth = b->coll_cloth;
        p.coll_count = &b->ctrl->coll_count;
        prm[i] = p;
        for (int sy = 0; sy < p.strips_y; sy++)
            for (int sx = 0; sx < p.strips_x; sx++) {
                const int cols = std::min(scols, p.nx - sx * scols);
                const int rows = std::min(p.rows_per_warp, p.ny - sy * p.rows_per_warp);
                items.push_back(make_int4((int)i, sx, sy, cols * rows));
            }
    }
    std::stable_sort(items.begin(), items.end(), [](const int4 &a, const int4 &c) { return a.w > c.w; });
    cudaFree(b->d_params);
    cudaFree(b->d_items);
    b->d_params = nullptr;
    b->d_items = nullptr;
    cudaError_t e = cudaMalloc(&b->d_params, sizeof(StepParams) * prm.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_params, prm.data(), sizeof(StepParams) * prm.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->n_items = (int)items.size();
    b->args.params = b->d_params;
    b->args.items = b->d_items;
    b->args.n_items = b->n_items;
    b->args.work = b->work;
    b->args.ctrl = b->ctrl;
    b->args.coll_list = b->coll_list;
    b->args.coll_cloth = b->coll_cloth;
    b->args.coll_count = &b->ctrl->coll_count;
    b->args.walk_blocks = b->sm_count * b->ctas_per_sm;
    b->args.coll_blocks = b->sm_count * CLOTH_COLL_CTAS_PER_SM;
    // one walk variant for the whole batch when every cloth has the same one
    int var = -1;
    for (const StepParams &q : prm) {
        const int v = (q.has_mesh ? BATCH_VAR_MESH : 0) | (q.ks_slot ? BATCH_VAR_PER_SPRING : 0);
        var = var < 0 || var == v ? v : BATCH_VAR_MIXED;
    }
    b->args.variant = var < 0 ? BATCH_VAR_MIXED : var;
    return e;
}

cudaError_t ensure_graph(ClothBatch *b)
{
    if (b->graph) return cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < b->substeps && le == cudaSuccess; s++) le = launch_batch_substep(b->args, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    return e;
}

void free_batch(ClothBatch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (ClothHandle *h : b->cl) cloth_destroy(h);
    b->cl.clear();
    cudaFree(b->ctrl);
    cudaFree(b->work);
    cudaFree(b->coll_list);
    cudaFree(b->coll_cloth);
    cudaFree(b->d_params);
    cudaFree(b->d_items);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

int read_batch_flags(ClothBatch *b)
{
    unsigned flags = 0;
    BTRY(b, cudaMemcpyAsync(&flags, &b->ctrl->flags, sizeof(flags), cudaMemcpyDeviceToHost, b->stream),
         "read flags");
    BTRY(b, cudaStreamSynchronize(b->stream), "synchronize");
    if (flags & CTRL_FLAG_TIMEOUT) return bfail(CLOTH_ERR_TIMEOUT, "a device-side wait timed out");
    if (flags & CTRL_FLAG_NONFINITE) return bfail(CLOTH_ERR_NONFINITE, "a cloth of the batch became non-finite");
    return CLOTH_OK;
}

}  // namespace

extern "C" {

int cloth_batch_create(const ClothDesc *descs, int32_t count, void *stream, ClothBatch **out)
{
    if (!out) return bfail(CLOTH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || count < 1) return bfail(CLOTH_ERR_INVALID_ARG, "need at least one description");
    for (int i = 0; i < count; i++)
        if (descs[i].flags & (CLOTH_FLAG_ATOMIC_SPRINGS | CLOTH_FLAG_EDGE_COLLISION))
            return bfail(CLOTH_ERR_INVALID_ARG,
                         "CLOTH_FLAG_ATOMIC_SPRINGS and CLOTH_FLAG_EDGE_COLLISION are not supported in batches");
    for (int i = 1; i < count; i++)
        if (descs[i].dt != descs[0].dt || descs[i].substeps != descs[0].substeps)
            return bfail(CLOTH_ERR_INVALID_ARG, "every cloth of a batch needs the same dt and substeps (cloth %d)", i);
    ClothBatch *b = new (std::nothrow) ClothBatch();
    if (!b) return bfail(CLOTH_ERR_OOM, "host allocation failed");
    b->stream = (cudaStream_t)stream;
    b->substeps = descs[0].substeps;
    cudaGetDevice(&b->device);
    if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        b->sm_count < 1)
        b->sm_count = 152;
    cudaGetLastError();
    b->ctas_per_sm = batch_min_ctas();
    long long total = 0;
    try {
        b->cl.reserve((size_t)count);
        for (int i = 0; i < count; i++) {
            ClothHandle *h = nullptr;
            int rc = cloth_create(&descs[i], stream, &h);
            if (rc) {
                free_batch(b);
                delete b;
                return rc;
            }
            b->cl.push_back(h);
            total += h->n;
        }
    } catch (...) {
        free_batch(b);
        delete b;
        return bfail(CLOTH_ERR_OOM, "host allocation failed");
    }
    // a default strip height from the whole batch's rows: about one wave of warps
    long long strips_x_rows = 0;
    for (ClothHandle *h : b->cl)
        strips_x_rows += (long long)((h->desc.nx + substep_strip_cols() - 1) / substep_strip_cols()) * h->desc.ny;
    const long long warps = (long long)b->sm_count * substep_warps_per_cta() * b->ctas_per_sm;
    long long R = (strips_x_rows + warps - 1) / warps;
    b->rows_per_warp = (int)std::min<long long>(CLOTH_MAX_ROWS_PER_WARP, std::max<long long>(4, R));
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->ctrl, sizeof(DevCtrl));
    if (e == cudaSuccess) e = cudaMalloc(&b->work, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->coll_list, sizeof(int) * (size_t)total);
    if (e == cudaSuccess) e = cudaMalloc(&b->coll_cloth, sizeof(int) * (size_t)total);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctrl, 0, sizeof(DevCtrl), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->work, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) {
        try {
            e = rebuild(b);
        } catch (...) {
            e = cudaErrorMemoryAllocation;
        }
    }
    if (e != cudaSuccess) {
        int rc = e == cudaErrorMemoryAllocation ? bfail(CLOTH_ERR_OOM, "device allocation failed")
                                                 : bcuda(nullptr, e, "cloth_batch_create");
        free_batch(b);
        delete b;
        cudaGetLastError();
        return rc;
    }
    *out = b;
    return CLOTH_OK;
}

int cloth_batch_set_mesh(ClothBatch *b, int32_t index, const float *verts, int32_t nverts, const int32_t *tris,
                         int32_t ntris)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (index < 0 || index >= (int)b->cl.size()) return bfail(CLOTH_ERR_INVALID_ARG, "cloth index %d", index);
    rc = cloth_set_mesh(b->cl[index], verts, nverts, tris, ntris);
    if (rc) return rc;
    try {
        BTRY(b, rebuild(b), "batch rebuild");
    } catch (...) {
        return bfail(CLOTH_ERR_OOM, "host allocation failed");
    }
    return CLOTH_OK;
}

int cloth_batch_step(ClothBatch *b, int32_t nsteps)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (nsteps < 0) return bfail(CLOTH_ERR_INVALID_ARG, "nsteps < 0");
    BTRY(b, ensure_graph(b), "graph capture");
    for (int s = 0; s < nsteps; s++) BTRY(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
    b->substeps_done += (long long)nsteps * b->substeps;
    return CLOTH_OK;
}

int cloth_batch_read(ClothBatch *b, int32_t index, float *pos_out, float *vel_out)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (index < 0 || index >= (int)b->cl.size()) return bfail(CLOTH_ERR_INVALID_ARG, "cloth index %d", index);
    ClothHandle *h = b->cl[index];
    const long long N = h->n;
    if (pos_out || vel_out) {
        BTRY(b, launch_soa_to_aos(h->state, h->state + 6 * h->stride, h->stride, h->n, h->desc.nx, h->pitch, b->ctrl,
                                  pos_out ? h->staging : nullptr, vel_out ? h->staging + 3 * N : nullptr, b->stream),
             "state gather");
        if (pos_out)
            BTRY(b, cudaMemcpyAsync(pos_out, h->staging, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, b->stream),
                 "copy positions");
        if (vel_out)
            BTRY(b, cudaMemcpyAsync(vel_out, h->staging + 3 * N, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost,
                                    b->stream),
                 "copy velocities");
    }
    return read_batch_flags(b);
}

int cloth_batch_set_state(ClothBatch *b, int32_t index, const float *pos, const float *vel)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (index < 0 || index >= (int)b->cl.size()) return bfail(CLOTH_ERR_INVALID_ARG, "cloth index %d", index);
    if (!pos && !vel) return CLOTH_OK;
    ClothHandle *h = b->cl[index];
    const long long N = h->n;
    if (pos)
        BTRY(b, cudaMemcpyAsync(h->staging, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, b->stream),
             "upload positions");
    if (vel)
        BTRY(b, cudaMemcpyAsync(h->staging + 3 * N, vel, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, b->stream),
             "upload velocities");
    BTRY(b, launch_aos_to_soa(pos ? h->staging : nullptr, vel ? h->staging + 3 * N : nullptr, h->state,
                              h->state + 6 * h->stride, h->stride, h->n, h->desc.nx, h->pitch, b->ctrl, b->stream),
         "state scatter");
    return CLOTH_OK;
}

int cloth_batch_set_tuning(ClothBatch *b, int32_t rows_per_warp, int32_t walk_ctas_per_sm)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (rows_per_warp < 1 || rows_per_warp > CLOTH_MAX_ROWS_PER_WARP || walk_ctas_per_sm < 1 ||
        walk_ctas_per_sm > 32)
        return bfail(CLOTH_ERR_INVALID_ARG, "rows_per_warp in [1,32], walk_ctas_per_sm in [1,32]");
    b->rows_per_warp = rows_per_warp;
    b->ctas_per_sm = walk_ctas_per_sm;
    try {
        BTRY(b, rebuild(b), "batch rebuild");
    } catch (...) {
        return bfail(CLOTH_ERR_OOM, "host allocation failed");
    }
    return CLOTH_OK;
}

int cloth_batch_tune(ClothBatch *b, int32_t trial_substeps, ClothBatchTuning *out)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (trial_substeps < 1 || !out) return bfail(CLOTH_ERR_INVALID_ARG, "trial_substeps >= 1 and out required");
    // save every state buffer and the control block; trials advance them
    std::vector<float *> saved(b->cl.size(), nullptr);
    DevCtrl ctrl_saved;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best_R = b->rows_per_warp, best_c = b->ctas_per_sm, tried = 0;
    float best_us = INFINITY;
    cudaError_t e = cudaMemcpyAsync(&ctrl_saved, b->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, b->stream);
    for (size_t i = 0; i < b->cl.size() && e == cudaSuccess; i++) {
        ClothHandle *h = b->cl[i];
        e = cudaMalloc(&saved[i], sizeof(float) * 12 * (size_t)h->stride);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(saved[i], h->state, sizeof(float) * 12 * (size_t)h->stride, cudaMemcpyDeviceToDevice,
                                b->stream);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int Rs[] = {4, 6, 8, 12, 16, 24, 32};
    for (int c = 1; c <= batch_min_ctas() && e == cudaSuccess; c++)
        for (int R : Rs) {
            if (e != cudaSuccess) break;
            b->rows_per_warp = R;
            b->ctas_per_sm = c;
            try {
                e = rebuild(b);
            } catch (...) {
                e = cudaErrorMemoryAllocation;
            }
            if (e == cudaSuccess) e = launch_batch_substep(b->args, b->stream);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int s = 0; s < trial_substeps && e == cudaSuccess; s++) e = launch_batch_substep(b->args, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) {
                tried++;
                const float us = 1e3f * ms / (float)trial_substeps;
                if (us < best_us) {
                    best_us = us;
                    best_R = R;
                    best_c = c;
                }
            }
        }
    // restore the states and the counter, then apply the winner
    for (size_t i = 0; i < b->cl.size(); i++) {
        ClothHandle *h = b->cl[i];
        if (saved[i] && e == cudaSuccess)
            e = cudaMemcpyAsync(h->state, saved[i], sizeof(float) * 12 * (size_t)h->stride, cudaMemcpyDeviceToDevice,
                                b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ctrl, &ctrl_saved, sizeof(DevCtrl), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    for (float *p : saved) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return bcuda(b, e, "batch tuning");
    b->rows_per_warp = best_R;
    b->ctas_per_sm = best_c;
    try {
        BTRY(b, rebuild(b), "batch rebuild");
    } catch (...) {
        return bfail(CLOTH_ERR_OOM, "host allocation failed");
    }
    out->rows_per_warp = best_R;
    out->walk_ctas_per_sm = best_c;
    out->us_per_substep = best_us;
    out->candidates = tried;
    return CLOTH_OK;
}

int cloth_batch_get_tuning(ClothBatch *b, ClothBatchTuning *out)
{
    int rc = check_batch(b);
    if (rc) return rc;
    if (!out) return bfail(CLOTH_ERR_INVALID_ARG, "out is NULL");
    out->rows_per_warp = b->rows_per_warp;
    out->walk_ctas_per_sm = b->ctas_per_sm;
    out->us_per_substep = 0.0f;
    out->candidates = 0;
    return CLOTH_OK;
}

int cloth_batch_sync(ClothBatch *b)
{
    int rc = check_batch(b);
    if (rc) return rc;
    return read_batch_flags(b);
}

int cloth_batch_get_collision_stats(ClothBatch *b, int64_t *listed, int64_t *tested, int64_t *hits)
{
    int rc = check_batch(b);
    if (rc) return rc;
    unsigned long long v[3] = {0ull, 0ull, 0ull};
    BTRY(b, cudaMemcpyAsync(v, &b->ctrl->stat_listed, sizeof(v), cudaMemcpyDeviceToHost, b->stream),
         "read collision statistics");
    BTRY(b, cudaStreamSynchronize(b->stream), "synchronize");
    if (listed) *listed = (int64_t)v[0];
    if (tested) *tested = (int64_t)v[1];
    if (hits) *hits = (int64_t)v[2];
    return CLOTH_OK;
}

void cloth_batch_destroy(ClothBatch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
