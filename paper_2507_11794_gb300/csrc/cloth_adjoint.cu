// Reverse mode of the cloth step (not in the paper): gradients of a loss on
// the final state w.r.t. per-spring stiffness and damping and the initial
// velocities, with the contact set of every substep frozen at the one the
// forward pass found.  A rollout runs the forward pass keeping a checkpoint
// every `checkpoint_every` steps; the backward pass recomputes one segment at
// a time (storing each substep's start state and post-integration velocity)
// and walks it in reverse:
//   response   x' = S + m r (contact: m = mean max(t_k - delta, 0) over the
//              hits, r = v*/|v*|, v' = c v*) or x' = S + dt v*, v' = v*;
//   Euler      v* = v + dt (F/m + g + w);
//   springs    Algorithm 1's force, differentiated in x, v, ks, kd; each node
//              gathers its twelve springs, each spring's owner alone writes
//              its ks/kd gradient (no atomics, fixed order).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <new>
#include <vector>

#include "cloth_collide.cuh"
#include "cloth_internal.h"

namespace {

// Canonical spring directions (drow, dcol).
constexpr int DR[CLOTH_NDIR] = {0, 1, 1, 1, 0, 2};
constexpr int DC[CLOTH_NDIR] = {1, 0, 1, -1, 2, 0};
__device__ __forceinline__ int dev_dr(int d) { return d == 0 || d == 4 ? 0 : (d == 5 ? 2 : 1); }
__device__ __forceinline__ int dev_dc(int d) { return d == 0 ? 1 : (d == 1 || d == 5 ? 0 : (d == 2 ? 1 : (d == 3 ? -1 : 2))); }

// Reverse of the response and the Euler update of one substep, one thread
// per node.  xs: 6 planes (x, v at the substep's start), vs: 3 planes (v*),
// lx/lv: adjoints of the substep's end; outputs lS (x part), lvp (v* part)
// and lF = dt/m lvp (force adjoint; 0 for pinned nodes).
__global__ void adj_contact_kernel(const StepParams p, const float *__restrict__ xs, const float *__restrict__ vs,
                                   const float *__restrict__ lx, const float *__restrict__ lv, float *__restrict__ lS,
                                   float *__restrict__ lvp, float *__restrict__ lF)
{
    const long long st = p.stride;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)p.ny * p.pitch) return;
    const int c = (int)(idx % p.pitch);
    if (c >= p.nx) return;
    const long long o = idx;
    const float l0 = lx[o], l1 = lx[st + o], l2 = lx[2 * st + o];
    const bool pinned = p.pin_bits && ((p.pin_bits[o >> 5] >> (o & 31)) & 1u);
    if (pinned) {
        lS[o] = l0; lS[st + o] = l1; lS[2 * st + o] = l2;
        lvp[o] = lvp[st + o] = lvp[2 * st + o] = 0.0f;
        lF[o] = lF[st + o] = lF[2 * st + o] = 0.0f;
        return;
    }
    const float m0 = lv[o], m1 = lv[st + o], m2 = lv[2 * st + o];
    const float sx = xs[o], sy = xs[st + o], sz = xs[2 * st + o];
    const float wx = vs[o], wy = vs[st + o], wz = vs[2 * st + o];
    // the predicted end exactly as the forward pass formed it
    const float ex = fmaf(p.dt, wx, sx), ey = fmaf(p.dt, wy, sy), ez = fmaf(p.dt, wz, sz);
    float s0 = l0, s1 = l1, s2 = l2;
    float q0 = fmaf(p.dt, l0, m0), q1 = fmaf(p.dt, l1, m1), q2 = fmaf(p.dt, l2, m2);
    if (p.has_mesh) {
        float ox, oy, oz, g1[3] = {0.0f, 0.0f, 0.0f}, g2[3] = {0.0f, 0.0f, 0.0f}, mK[5];
        if (collide_t<true>(p, sx, sy, sz, ex, ey, ez, ox, oy, oz, g1, g2, mK)) {
            const float m = mK[0], invK = 1.0f / mK[1], rx = mK[2], ry = mK[3], rz = mK[4];
            const float rl = rx * l0 + ry * l1 + rz * l2;
            s0 = l0 + g1[0] * invK * rl;
            s1 = l1 + g1[1] * invK * rl;
            s2 = l2 + g1[2] * invK * rl;
            const float r0 = m * l0 + g2[0] * invK * rl, r1 = m * l1 + g2[1] * invK * rl,
                        r2 = m * l2 + g2[2] * invK * rl;
            const float rr = rx * r0 + ry * r1 + rz * r2;
            const float inv_nv = rsqrtf(wx * wx + wy * wy + wz * wz);
            q0 = (r0 - rx * rr) * inv_nv + p.restitution * m0;
            q1 = (r1 - ry * rr) * inv_nv + p.restitution * m1;
            q2 = (r2 - rz * rr) * inv_nv + p.restitution * m2;
        }
    }
    lS[o] = s0; lS[st + o] = s1; lS[2 * st + o] = s2;
    lvp[o] = q0; lvp[st + o] = q1; lvp[2 * st + o] = q2;
    const float sc = p.dt * p.inv_mass;
    lF[o] = sc * q0; lF[st + o] = sc * q1; lF[2 * st + o] = sc * q2;
}

// Adjoint of one spring seen from its owner o (forward spring o -> e):
// mu = lF_o - lF_e; returns gd = (dF/dd)^T mu, gv = (dF/ddv)^T mu and the
// ks / kd gradient terms.
__device__ __forceinline__ void spring_adj(const float *xo, const float *vo, const float *xe, const float *ve,
                                           const float *mu, float ks, float kd, float L0, float gd[3], float gv[3],
                                           float &gks, float &gkd)
{
    const float dx = xe[0] - xo[0], dy = xe[1] - xo[1], dz = xe[2] - xo[2];
    const float l2 = dx * dx + dy * dy + dz * dz;
    gd[0] = gd[1] = gd[2] = gv[0] = gv[1] = gv[2] = 0.0f;
    gks = gkd = 0.0f;
    if (!(l2 > 1e-24f)) return;
    const float il = rsqrtf(l2), l = l2 * il;
    const float ux = dx * il, uy = dy * il, uz = dz * il;
    const float dvx = ve[0] - vo[0], dvy = ve[1] - vo[1], dvz = ve[2] - vo[2];
    const float ud = ux * dvx + uy * dvy + uz * dvz;
    const float um = ux * mu[0] + uy * mu[1] + uz * mu[2];
    const float phi = ks * (l - L0) + kd * ud;
    const float a = phi * il, b = kd * il;
    gd[0] = a * (mu[0] - ux * um) + um * (ks * ux + b * (dvx - ux * ud));
    gd[1] = a * (mu[1] - uy * um) + um * (ks * uy + b * (dvy - uy * ud));
    gd[2] = a * (mu[2] - uz * um) + um * (ks * uz + b * (dvz - uz * ud));
    gv[0] = kd * ux * um;
    gv[1] = kd * uy * um;
    gv[2] = kd * uz * um;
    gks = um * (l - L0);
    gkd = um * ud;
}

// Reverse of the spring forces, one thread per node: the node's adjoints of
// the substep's start state (lx, lv) and += gradients of the springs it owns.
__global__ void adj_spring_kernel(const StepParams p, const float *__restrict__ xs, const float *__restrict__ lF,
                                  const float *__restrict__ lS, const float *__restrict__ lvp, float *__restrict__ lx,
                                  float *__restrict__ lv, double *__restrict__ gks, double *__restrict__ gkd)
{
    const long long st = p.stride;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)p.ny * p.pitch) return;
    const int r = (int)(idx / p.pitch), c = (int)(idx % p.pitch);
    if (c >= p.nx) return;
    const long long o = idx;
    const float xi[3] = {xs[o], xs[st + o], xs[2 * st + o]};
    const float vi[3] = {xs[3 * st + o], xs[4 * st + o], xs[5 * st + o]};
    const float fi[3] = {lF[o], lF[st + o], lF[2 * st + o]};
    float gx[3] = {lS[o], lS[st + o], lS[2 * st + o]};
    float gv[3] = {lvp[o], lvp[st + o], lvp[2 * st + o]};
#pragma unroll
    for (int d = 0; d < CLOTH_NDIR; d++) {
        // spring owned by this node
        {
            const int r2 = r + dev_dr(d), c2 = c + dev_dc(d);
            if (r2 < p.ny && c2 >= 0 && c2 < p.nx) {
                const long long e = (long long)r2 * p.pitch + c2;
                const float xe[3] = {xs[e], xs[st + e], xs[2 * st + e]};
                const float ve[3] = {xs[3 * st + e], xs[4 * st + e], xs[5 * st + e]};
                const float mu[3] = {fi[0] - lF[e], fi[1] - lF[st + e], fi[2] - lF[2 * st + e]};
                float a[3], b[3], g1, g2;
                spring_adj(xi, vi, xe, ve, mu, p.ks_slot[d * st + o], p.kd_slot[d * st + o], p.L0[d], a, b, g1, g2);
                gx[0] -= a[0]; gx[1] -= a[1]; gx[2] -= a[2];
                gv[0] -= b[0]; gv[1] -= b[1]; gv[2] -= b[2];
                // per-spring sums over the substeps in double: FP64 only in these reductions
                gks[d * st + o] += (double)g1;
                gkd[d * st + o] += (double)g2;
            }
        }
        // spring owned by the node at (-dr, -dc), ending here
        {
            const int r2 = r - dev_dr(d), c2 = c - dev_dc(d);
            if (r2 >= 0 && c2 >= 0 && c2 < p.nx) {
                const long long w = (long long)r2 * p.pitch + c2;
                const float xw[3] = {xs[w], xs[st + w], xs[2 * st + w]};
                const float vw[3] = {xs[3 * st + w], xs[4 * st + w], xs[5 * st + w]};
                const float mu[3] = {lF[w] - fi[0], lF[st + w] - fi[1], lF[2 * st + w] - fi[2]};
                float a[3], b[3], g1, g2;
                spring_adj(xw, vw, xi, vi, mu, p.ks_slot[d * st + w], p.kd_slot[d * st + w], p.L0[d], a, b, g1, g2);
                gx[0] += a[0]; gx[1] += a[1]; gx[2] += a[2];
                gv[0] += b[0]; gv[1] += b[1]; gv[2] += b[2];
            }
        }
    }
    lx[o] = gx[0]; lx[st + o] = gx[1]; lx[2 * st + o] = gx[2];
    lv[o] = gv[0]; lv[st + o] = gv[1]; lv[2 * st + o] = gv[2];
}

// Canonical spring order <-> [direction][r*pitch + c] slots.
__global__ void scatter_kernel(const float *__restrict__ canon, const int *__restrict__ map, int S,
                               float *__restrict__ slot)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) slot[map[s]] = canon[s];
}
__global__ void gather_kernel(const double *__restrict__ slot, const int *__restrict__ map, int S,
                              float *__restrict__ canon)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) canon[s] = (float)slot[map[s]];
}
// AoS [N][3] <-> three planes of the pitch layout.
__global__ void aos_planes_kernel(const float *__restrict__ aos, int n, int nx, int pitch, long long st,
                                  float *__restrict__ planes)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long o = (long long)(i / nx) * pitch + (i % nx);
    planes[o] = aos ? aos[3 * (long long)i] : 0.0f;
    planes[st + o] = aos ? aos[3 * (long long)i + 1] : 0.0f;
    planes[2 * st + o] = aos ? aos[3 * (long long)i + 2] : 0.0f;
}
__global__ void planes_aos_kernel(const float *__restrict__ planes, int n, int nx, int pitch, long long st,
                                  float *__restrict__ aos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long o = (long long)(i / nx) * pitch + (i % nx);
    aos[3 * (long long)i] = planes[o];
    aos[3 * (long long)i + 1] = planes[st + o];
    aos[3 * (long long)i + 2] = planes[2 * st + o];
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

struct ClothRollout {
    ClothHandle *h = nullptr;
    int nsteps = 0, every = 0, nseg = 0, S = 0;
    unsigned long long k0 = 0, k_final = 0;
    std::vector<unsigned long long> kseg;  // substep counter at each checkpoint (host copies for async uploads)
    float *x0 = nullptr, *v0 = nullptr;    // initial state, AoS [N][3]
    float *ckpt = nullptr;                 // nseg x 6 planes
    float *seg = nullptr;                  // every*substeps x 9 planes (x, v, v*)
    float *lam = nullptr;                  // lx, lv, lS, lvp, lF: 15 planes
    double *gslot = nullptr;               // gks, gkd: 12 planes (double sums over substeps)
    float *final_state = nullptr;          // 6 planes
    int *map = nullptr;                    // canonical spring -> slot
    bool forward_done = false;
};

namespace {

int rfail(int code, const char *fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    cloth_set_error_message(msg);
    return code;
}

#define RTRY(h, call, what)                                                                                       \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) {                                                                                  \
            (h)->dead = true;                                                                                     \
            return rfail(CLOTH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e_), cudaGetErrorString(e_));      \
        }                                                                                                         \
    } while (0)

float *cur_state(ClothHandle *h, unsigned long long k) { return h->state + ((k & 1ull) ? 6 * h->stride : 0); }

}  // namespace

extern "C" {

int cloth_rollout_create(ClothHandle *h, int32_t nsteps, int32_t checkpoint_every, ClothRollout **out)
{
    if (!out) return rfail(CLOTH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!h) return rfail(CLOTH_ERR_INVALID_ARG, "null handle");
    if (h->dead) return rfail(CLOTH_ERR_STATE, "handle unusable after an earlier CUDA error");
    if (nsteps < 1 || checkpoint_every < 1) return rfail(CLOTH_ERR_INVALID_ARG, "nsteps and checkpoint_every >= 1");
    // the reverse pass recomputes each segment and must see the forward pass's
    // exact states (the atomic path is not bitwise reproducible) and its
    // node-path contacts
    if (h->desc.flags & (CLOTH_FLAG_EDGE_COLLISION | CLOTH_FLAG_ATOMIC_SPRINGS))
        return rfail(CLOTH_ERR_INVALID_ARG,
                     "rollouts need the default path (no CLOTH_FLAG_EDGE_COLLISION or CLOTH_FLAG_ATOMIC_SPRINGS)");
    const ClothDesc &d = h->desc;
    const long long N = h->n, st = h->stride;
    ClothRollout *ro = new (std::nothrow) ClothRollout();
    if (!ro) return rfail(CLOTH_ERR_OOM, "host allocation failed");
    ro->h = h;
    ro->nsteps = nsteps;
    ro->every = checkpoint_every < nsteps ? checkpoint_every : nsteps;
    ro->nseg = (nsteps + ro->every - 1) / ro->every;
    ro->k0 = (unsigned long long)h->substeps_done;
    cudaError_t e = cudaSuccess;
    std::vector<int> map;
    std::vector<float> ks, kd;
    try {
        ro->kseg.resize((size_t)ro->nseg + 2);
        // canonical order -> slot index, and per-type constants for missing slots
        const int type[CLOTH_NDIR] = {0, 0, 1, 1, 2, 2};
        for (long long r = 0; r < d.ny; r++)
            for (long long c = 0; c < d.nx; c++)
                for (int k = 0; k < CLOTH_NDIR; k++) {
                    const long long r2 = r + DR[k], c2 = c + DC[k];
                    if (r2 < 0 || r2 >= d.ny || c2 < 0 || c2 >= d.nx) continue;
                    map.push_back((int)(k * st + r * h->pitch + c));
                    ks.push_back(d.ks[type[k]]);
                    kd.push_back(d.kd[type[k]]);
                }
    } catch (...) {
        delete ro;
        return rfail(CLOTH_ERR_OOM, "host allocation failed");
    }
    ro->S = (int)map.size();
    const size_t seg_sub = (size_t)ro->every * d.substeps;
    if (e == cudaSuccess) e = cudaMalloc(&ro->x0, sizeof(float) * 3 * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc(&ro->v0, sizeof(float) * 3 * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc(&ro->ckpt, sizeof(float) * 6 * (size_t)st * (size_t)ro->nseg);
    if (e == cudaSuccess) e = cudaMalloc(&ro->seg, sizeof(float) * 9 * (size_t)st * seg_sub);
    if (e == cudaSuccess) e = cudaMalloc(&ro->lam, sizeof(float) * 15 * (size_t)st);
    if (e == cudaSuccess) e = cudaMalloc(&ro->gslot, sizeof(double) * 12 * (size_t)st);
    if (e == cudaSuccess) e = cudaMalloc(&ro->final_state, sizeof(float) * 6 * (size_t)st);
    if (e == cudaSuccess) e = cudaMalloc(&ro->map, sizeof(int) * (size_t)(ro->S > 0 ? ro->S : 1));
    if (e == cudaSuccess && ro->S > 0)
        e = cudaMemcpy(ro->map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h->ks_slot) {
        // the rollout differentiates per spring: give the cloth per-spring planes
        if ((e = cudaMalloc(&h->ks_slot, sizeof(float) * 6 * (size_t)st)) == cudaSuccess &&
            (e = cudaMalloc(&h->kd_slot, sizeof(float) * 6 * (size_t)st)) == cudaSuccess &&
            (e = cudaMemsetAsync(h->ks_slot, 0, sizeof(float) * 6 * (size_t)st, h->stream)) == cudaSuccess &&
            (e = cudaMemsetAsync(h->kd_slot, 0, sizeof(float) * 6 * (size_t)st, h->stream)) == cudaSuccess) {
            float *tmp = nullptr;
            if ((e = cudaMalloc(&tmp, sizeof(float) * (size_t)(ro->S > 0 ? ro->S : 1))) == cudaSuccess && ro->S > 0) {
                if ((e = cudaMemcpy(tmp, ks.data(), sizeof(float) * ks.size(), cudaMemcpyHostToDevice)) ==
                    cudaSuccess) {
                    scatter_kernel<<<nblk(ro->S, 256), 256, 0, h->stream>>>(tmp, ro->map, ro->S, h->ks_slot);
                    e = cudaMemcpyAsync(tmp, kd.data(), sizeof(float) * kd.size(), cudaMemcpyHostToDevice, h->stream);
                    if (e == cudaSuccess) {
                        // the copy above is ordered after the first scatter on the stream
                        scatter_kernel<<<nblk(ro->S, 256), 256, 0, h->stream>>>(tmp, ro->map, ro->S, h->kd_slot);
                        e = cudaStreamSynchronize(h->stream);
                    }
                }
            }
            cudaFree(tmp);
        }
        if (e == cudaSuccess) {
            cloth_fill_params(h);
            if (h->graph) cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
    }
    // the current state is the rollout's initial state
    if (e == cudaSuccess)
        e = launch_soa_to_aos(h->state, h->state + 6 * h->stride, h->stride, h->n, d.nx, h->pitch, h->ctrl, ro->x0,
                              ro->v0, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cloth_rollout_destroy(ro);
        return rfail(e == cudaErrorMemoryAllocation ? CLOTH_ERR_OOM : CLOTH_ERR_CUDA, "cloth_rollout_create: %s",
                     cudaGetErrorString(e));
    }
    *out = ro;
    return CLOTH_OK;
}

int cloth_rollout_forward(ClothRollout *ro, const float *d_ks, const float *d_kd, const float *d_v0, float *d_pos_out,
                          float *d_vel_out)
{
    if (!ro || !ro->h) return rfail(CLOTH_ERR_INVALID_ARG, "null rollout");
    ClothHandle *h = ro->h;
    if (h->dead) return rfail(CLOTH_ERR_STATE, "handle unusable after an earlier CUDA error");
    const long long st = h->stride;
    cudaStream_t s = h->stream;
    if (d_ks) scatter_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(d_ks, ro->map, ro->S, h->ks_slot);
    if (d_kd) scatter_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(d_kd, ro->map, ro->S, h->kd_slot);
    RTRY(h, cudaGetLastError(), "constants scatter");
    ro->kseg[0] = ro->k0;
    RTRY(h, cudaMemcpyAsync(&h->ctrl->k, &ro->kseg[0], sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
         "set substep counter");
    RTRY(h, launch_aos_to_soa(ro->x0, d_v0 ? d_v0 : ro->v0, h->state, h->state + 6 * st, st, h->n, h->desc.nx,
                              h->pitch, h->ctrl, s),
         "initial state");
    unsigned long long k = ro->k0;
    for (int g = 0; g < ro->nseg; g++) {
        ro->kseg[g] = k;
        RTRY(h, cudaMemcpyAsync(ro->ckpt + (size_t)g * 6 * st, cur_state(h, k), sizeof(float) * 6 * st,
                                cudaMemcpyDeviceToDevice, s),
             "checkpoint");
        const int steps = (g == ro->nseg - 1) ? ro->nsteps - g * ro->every : ro->every;
        for (int q = 0; q < steps * h->desc.substeps; q++) RTRY(h, launch_substep(h->params, s), "substep");
        k += (unsigned long long)steps * h->desc.substeps;
    }
    ro->k_final = k;
    h->substeps_done = (long long)k;
    RTRY(h, cudaMemcpyAsync(ro->final_state, cur_state(h, k), sizeof(float) * 6 * st, cudaMemcpyDeviceToDevice, s),
         "save final state");
    if (d_pos_out || d_vel_out)
        RTRY(h, launch_soa_to_aos(h->state, h->state + 6 * st, st, h->n, h->desc.nx, h->pitch, h->ctrl, d_pos_out,
                                  d_vel_out, s),
             "final state");
    ro->forward_done = true;
    return CLOTH_OK;
}

int cloth_rollout_backward(ClothRollout *ro, const float *d_gpos, const float *d_gvel, float *d_gks, float *d_gkd,
                           float *d_gv0)
{
    if (!ro || !ro->h) return rfail(CLOTH_ERR_INVALID_ARG, "null rollout");
    ClothHandle *h = ro->h;
    if (h->dead) return rfail(CLOTH_ERR_STATE, "handle unusable after an earlier CUDA error");
    if (!ro->forward_done) return rfail(CLOTH_ERR_INVALID_ARG, "cloth_rollout_backward before forward");
    const long long st = h->stride;
    const int n = h->n, nx = h->desc.nx, sub = h->desc.substeps;
    cudaStream_t s = h->stream;
    float *lx = ro->lam, *lv = ro->lam + 3 * st, *lS = ro->lam + 6 * st, *lvp = ro->lam + 9 * st,
          *lF = ro->lam + 12 * st;
    const long long total = (long long)h->desc.ny * h->pitch;
    RTRY(h, cudaMemsetAsync(ro->lam, 0, sizeof(float) * 15 * st, s), "clear adjoints");
    RTRY(h, cudaMemsetAsync(ro->gslot, 0, sizeof(double) * 12 * st, s), "clear gradients");
    aos_planes_kernel<<<nblk(n, 256), 256, 0, s>>>(d_gpos, n, nx, h->pitch, st, lx);
    aos_planes_kernel<<<nblk(n, 256), 256, 0, s>>>(d_gvel, n, nx, h->pitch, st, lv);
    RTRY(h, cudaGetLastError(), "load output adjoints");
    StepParams p = h->params;
    for (int g = ro->nseg - 1; g >= 0; g--) {
        const int steps = (g == ro->nseg - 1) ? ro->nsteps - g * ro->every : ro->every;
        const int nsub = steps * sub;
        const unsigned long long kg = ro->kseg[g];
        // restore the checkpoint and recompute the segment, keeping every
        // substep's start state and post-integration velocity
        RTRY(h, cudaMemcpyAsync(&h->ctrl->k, &ro->kseg[g], sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
             "set substep counter");
        RTRY(h, cudaMemcpyAsync(cur_state(h, kg), ro->ckpt + (size_t)g * 6 * st, sizeof(float) * 6 * st,
                                cudaMemcpyDeviceToDevice, s),
             "restore checkpoint");
        for (int j = 0; j < nsub; j++) {
            float *sj = ro->seg + (size_t)j * 9 * st;
            RTRY(h, cudaMemcpyAsync(sj, cur_state(h, kg + j), sizeof(float) * 6 * st, cudaMemcpyDeviceToDevice, s),
                 "store substep state");
            StepParams q = p;
            q.vstar = sj + 6 * st;
            RTRY(h, launch_substep(q, s), "recompute substep");
        }
        for (int j = nsub - 1; j >= 0; j--) {
            const float *sj = ro->seg + (size_t)j * 9 * st;
            adj_contact_kernel<<<nblk(total, 256), 256, 0, s>>>(p, sj, sj + 6 * st, lx, lv, lS, lvp, lF);
            adj_spring_kernel<<<nblk(total, 256), 256, 0, s>>>(p, sj, lF, lS, lvp, lx, lv, ro->gslot,
                                                               ro->gslot + 6 * st);
            RTRY(h, cudaGetLastError(), "reverse substep");
        }
    }
    if (d_gv0) planes_aos_kernel<<<nblk(n, 256), 256, 0, s>>>(lv, n, nx, h->pitch, st, d_gv0);
    if (d_gks) gather_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(ro->gslot, ro->map, ro->S, d_gks);
    if (d_gkd) gather_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(ro->gslot + 6 * st, ro->map, ro->S, d_gkd);
    RTRY(h, cudaGetLastError(), "gradient outputs");
    // leave the cloth in its final forward state
    RTRY(h, cudaMemcpyAsync(&h->ctrl->k, &ro->k_final, sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
         "set substep counter");
    RTRY(h, cudaMemcpyAsync(cur_state(h, ro->k_final), ro->final_state, sizeof(float) * 6 * st,
                            cudaMemcpyDeviceToDevice, s),
         "restore final state");
    return CLOTH_OK;
}

void cloth_rollout_destroy(ClothRollout *ro)
{
    if (!ro) return;
    if (ro->h) cudaStreamSynchronize(ro->h->stream);
    cudaFree(ro->x0);
    cudaFree(ro->v0);
    cudaFree(ro->ckpt);
    cudaFree(ro->seg);
    cudaFree(ro->lam);
    cudaFree(ro->gslot);
    cudaFree(ro->final_state);
    cudaFree(ro->map);
    cudaGetLastError();
    delete ro;
}

}  // extern "C"
