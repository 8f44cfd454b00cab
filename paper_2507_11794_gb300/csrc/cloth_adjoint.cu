// Reverse mode of the cloth step (not in the paper): gradients of a loss on
// the final state w.r.t. per-spring stiffness and damping and the initial
// velocities, with the contact set of every substep frozen at the one the
// forward pass found.  A rollout runs the forward pass keeping a checkpoint
// every `checkpoint_every` steps; the backward pass recomputes one segment at
// a time (storing each substep's start state, post-integration velocity and
// the response data of the nodes that hit) and walks it in reverse, the
// recompute of the next segment overlapping the reverse of the current one:
//   response   x' = S + m r (contact: m = mean max(t_k - delta, 0) over the
//              hits, r = v*/|v*|, v' = c v*) or x' = S + dt v*, v' = v*;
//   Euler      v* = v + dt (F/m + g + w);
//   springs    Algorithm 1's force, differentiated in x, v, ks, kd; each node
//              gathers its twelve springs (four lanes, three each), each
//              spring's owner alone writes its ks/kd gradient (no atomics,
//              fixed order).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <initializer_list>
#include <new>
#include <vector>

#include "cloth_internal.h"

namespace {

// The reverse kernels are launched with programmatic stream serialisation:
// a launch may start while its predecessor drains, and griddepcontrol.wait,
// before any global memory access, blocks until the predecessor has
// completed and its writes are visible.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Canonical spring directions (drow, dcol).
constexpr int DR[CLOTH_NDIR] = {0, 1, 1, 1, 0, 2};
constexpr int DC[CLOTH_NDIR] = {1, 0, 1, -1, 2, 0};
__device__ __forceinline__ int dev_dr(int d) { return d == 0 || d == 4 ? 0 : (d == 5 ? 2 : 1); }
__device__ __forceinline__ int dev_dc(int d) { return d == 0 ? 1 : (d == 1 || d == 5 ? 0 : (d == 2 ? 1 : (d == 3 ? -1 : 2))); }

// Reverse of the response and the Euler update of one substep at node o.
// xs: 6 planes (x, v at the substep's start), vs: 3 planes (v*), cd / cb:
// the response data the recompute's collision pass recorded for the nodes
// that hit (m, r, g1 / K, g2 / K; see coll_record) and their bits; l, m:
// adjoints of the node's end position and velocity; writes lS (x part), lvp
// (v* part) and lF = dt/m lvp (force adjoint; 0 for a pinned node).
__device__ __forceinline__ void contact_adj(const StepParams &p, const float *__restrict__ xs,
                                            const float *__restrict__ vs, const float *__restrict__ cd,
                                            const uint32_t *__restrict__ cb, long long o, const float l[3],
                                            const float mv[3], float *__restrict__ lS, float *__restrict__ lvp,
                                            float *__restrict__ lF)
{
    const long long st = p.stride;
    const float l0 = l[0], l1 = l[1], l2 = l[2];
    const bool pinned = p.pin_bits && ((p.pin_bits[o >> 5] >> (o & 31)) & 1u);
    if (pinned) {
        lS[o] = l0; lS[st + o] = l1; lS[2 * st + o] = l2;
        lvp[o] = lvp[st + o] = lvp[2 * st + o] = 0.0f;
        lF[o] = lF[st + o] = lF[2 * st + o] = 0.0f;
        return;
    }
    const float m0 = mv[0], m1 = mv[1], m2 = mv[2];
    float s0 = l0, s1 = l1, s2 = l2;
    float q0 = fmaf(p.dt, l0, m0), q1 = fmaf(p.dt, l1, m1), q2 = fmaf(p.dt, l2, m2);
    if (cb && ((cb[o >> 5] >> (o & 31)) & 1u)) {
        // x' = S + m r with r = v*/|v*|, v' = c v*: dx'/dS = I + r g1^T / K,
        // dx'/dr = m I + r g2^T / K (t_k of the active hits vary with S and r)
        const float wx = vs[o], wy = vs[st + o], wz = vs[2 * st + o];
        const float m = cd[o], rx = cd[st + o], ry = cd[2 * st + o], rz = cd[3 * st + o];
        const float a0 = cd[4 * st + o], a1 = cd[5 * st + o], a2 = cd[6 * st + o];
        const float b0 = cd[7 * st + o], b1 = cd[8 * st + o], b2 = cd[9 * st + o];
        const float rl = rx * l0 + ry * l1 + rz * l2;
        s0 = l0 + a0 * rl;
        s1 = l1 + a1 * rl;
        s2 = l2 + a2 * rl;
        const float r0 = m * l0 + b0 * rl, r1 = m * l1 + b1 * rl, r2 = m * l2 + b2 * rl;
        const float rr = rx * r0 + ry * r1 + rz * r2;
        const float inv_nv = rsqrtf(wx * wx + wy * wy + wz * wz);
        q0 = (r0 - rx * rr) * inv_nv + p.restitution * m0;
        q1 = (r1 - ry * rr) * inv_nv + p.restitution * m1;
        q2 = (r2 - rz * rr) * inv_nv + p.restitution * m2;
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

// Reverse of the spring forces of one substep at node (r, c), offset o, as
// lane q (0..3) of the node's group of four lanes: the lane takes springs
// u = q, q + 4, q + 8 of the node's twelve in the order (owned d, incoming d,
// owned d + 1, ...), so lanes 0 and 2 take owned springs and write their
// ks / kd gradients, lanes 1 and 3 incoming ones.  xs is the substep's start
// state, lF its force adjoints (all nodes).  Returns the lane's part of the
// adjoints of the node's start position (gx) and velocity (gv).  Loads are
// issued unconditionally (a missing neighbour reads the node itself) so that
// the lane's gathers overlap; a missing spring's terms are discarded.
__device__ __forceinline__ void spring_adj_lane(const StepParams &p, const float *__restrict__ xs,
                                                const float *__restrict__ lF, long long o, int r, int c, int q,
                                                double *__restrict__ gks, double *__restrict__ gkd, float gx[3],
                                                float gv[3])
{
    const long long st = p.stride;
    const float xi[3] = {xs[o], xs[st + o], xs[2 * st + o]};
    const float vi[3] = {xs[3 * st + o], xs[4 * st + o], xs[5 * st + o]};
    const float fi[3] = {lF[o], lF[st + o], lF[2 * st + o]};
    const bool own = (q & 1) == 0;
    float xn[3][3], vn[3][3], ln[3][3], ksn[3], kdn[3];
    double sk[3], sd[3];
    bool ok[3];
    int dd[3];
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const int d = (q >> 1) + 2 * t;
        dd[t] = d;
        const int r2 = own ? r + dev_dr(d) : r - dev_dr(d);
        const int c2 = own ? c + dev_dc(d) : c - dev_dc(d);
        ok[t] = r2 >= 0 && r2 < p.ny && c2 >= 0 && c2 < p.nx;
        const long long e = ok[t] ? (long long)r2 * p.pitch + c2 : o;
        xn[t][0] = xs[e]; xn[t][1] = xs[st + e]; xn[t][2] = xs[2 * st + e];
        vn[t][0] = xs[3 * st + e]; vn[t][1] = xs[4 * st + e]; vn[t][2] = xs[5 * st + e];
        ln[t][0] = lF[e]; ln[t][1] = lF[st + e]; ln[t][2] = lF[2 * st + e];
        const long long so = d * st + (own ? o : e);  // the spring's slot: its owner's offset
        ksn[t] = p.ks_slot[so];
        kdn[t] = p.kd_slot[so];
        sk[t] = own ? gks[so] : 0.0;
        sd[t] = own ? gkd[so] : 0.0;
    }
    gx[0] = gx[1] = gx[2] = gv[0] = gv[1] = gv[2] = 0.0f;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const int d = dd[t];
        float a[3], b[3], g1, g2;
        if (own) {
            const float mu[3] = {fi[0] - ln[t][0], fi[1] - ln[t][1], fi[2] - ln[t][2]};
            spring_adj(xi, vi, xn[t], vn[t], mu, ksn[t], kdn[t], p.L0[d], a, b, g1, g2);
            if (ok[t]) {
                gx[0] -= a[0]; gx[1] -= a[1]; gx[2] -= a[2];
                gv[0] -= b[0]; gv[1] -= b[1]; gv[2] -= b[2];
                // per-spring sums over the substeps in double: FP64 only in these reductions
                gks[d * st + o] = sk[t] + (double)g1;
                gkd[d * st + o] = sd[t] + (double)g2;
            }
        } else {
            const float mu[3] = {ln[t][0] - fi[0], ln[t][1] - fi[1], ln[t][2] - fi[2]};
            spring_adj(xn[t], vn[t], xi, vi, mu, ksn[t], kdn[t], p.L0[d], a, b, g1, g2);
            if (ok[t]) {
                gx[0] += a[0]; gx[1] += a[1]; gx[2] += a[2];
                gv[0] += b[0]; gv[1] += b[1]; gv[2] += b[2];
            }
        }
    }
}

// Buffers of one reverse launch (plane layout, stride p.stride).
struct AdjArgs {
    const float *xs_s;      // spring part: start state of substep j (6 planes)
    const float *lF_s;      // spring part: force adjoints of substep j
    const float *xs_c;      // contact part: start state of the substep it reverses (6 planes)
    const float *vs_c;      // contact part: that substep's v* (3 planes)
    const float *cd_c;      // contact part: that substep's recorded response data (10 planes)
    const uint32_t *cb_c;   // contact part: its hit bits (null without a mesh)
    float *lF_c;            // contact part: its force adjoints (never lF_s: neighbours read lF_s)
    float *lS, *lvp;        // the node's own parts: read by the spring part, then written by the contact part
    float *lx, *lv;         // contact only: the end-state adjoints read; spring only: start-state adjoints written
    double *gks, *gkd;      // per-spring gradient sums
};

// One reverse launch, four lanes per node.  SPRING: the spring reverse of
// substep j (the lanes' parts summed as lS + ((q0 + q1) + (q2 + q3))) gives
// the node's start-state adjoints; CONTACT: lane 0 then runs the response
// and Euler reverse of the substep before (of the substep given, without
// SPRING), which consumes them at once.  Reversing a segment of n substeps
// takes n + 1 launches: contact(n-1), then spring(j) + contact(j-1) for
// j = n-1..1, then spring(0).
constexpr int ADJ_THREADS = 128;
constexpr int ADJ_LANES = 4;  // lanes per node
template <bool SPRING, bool CONTACT>
__global__ void __launch_bounds__(ADJ_THREADS) adj_kernel(const StepParams p, const AdjArgs a)
{
    pdl_enter();
    const long long st = p.stride;
    const long long idx = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / ADJ_LANES;
    const int q = threadIdx.x % ADJ_LANES;
    // the group's four lanes share idx, so they leave or stay together
    if (idx >= (long long)p.ny * p.pitch) return;
    const int r = (int)(idx / p.pitch), c = (int)(idx % p.pitch);
    if (c >= p.nx) return;
    if (!SPRING && q != 0) return;
    const long long o = idx;
    float l[3], m[3];
    if (SPRING) {
        const unsigned gm = 0xFu << (threadIdx.x & 28u);  // the group's lanes
        spring_adj_lane(p, a.xs_s, a.lF_s, o, r, c, q, a.gks, a.gkd, l, m);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            l[k] += __shfl_xor_sync(gm, l[k], 1);
            m[k] += __shfl_xor_sync(gm, m[k], 1);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            l[k] += __shfl_xor_sync(gm, l[k], 2);
            m[k] += __shfl_xor_sync(gm, m[k], 2);
        }
        if (q != 0) return;
        l[0] = a.lS[o] + l[0]; l[1] = a.lS[st + o] + l[1]; l[2] = a.lS[2 * st + o] + l[2];
        m[0] = a.lvp[o] + m[0]; m[1] = a.lvp[st + o] + m[1]; m[2] = a.lvp[2 * st + o] + m[2];
    } else {
        l[0] = a.lx[o]; l[1] = a.lx[st + o]; l[2] = a.lx[2 * st + o];
        m[0] = a.lv[o]; m[1] = a.lv[st + o]; m[2] = a.lv[2 * st + o];
    }
    if (CONTACT) {
        contact_adj(p, a.xs_c, a.vs_c, a.cd_c, a.cb_c, o, l, m, a.lS, a.lvp, a.lF_c);
    } else {
        a.lx[o] = l[0]; a.lx[st + o] = l[1]; a.lx[2 * st + o] = l[2];
        a.lv[o] = m[0]; a.lv[st + o] = m[1]; a.lv[2 * st + o] = m[2];
    }
}

// n floats (a multiple of 4, 16-byte aligned ends) from src to dst.
__global__ void copy_planes_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst, long long n4)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
// Start of a segment's recompute: the substep counter, and the hit bits of
// all its substeps cleared.
__global__ void segment_begin_kernel(DevCtrl *ctrl, unsigned long long k, uint32_t *bits, long long nwords)
{
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) ctrl->k = k;
    for (long long i = i0; i < nwords; i += (long long)gridDim.x * blockDim.x) bits[i] = 0u;
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

// Planes of one recompute slot: x, v (3 + 3), v* (3), response data (10).
constexpr int SLOT_PLANES = 19;

}  // namespace

struct ClothRollout {
    ClothHandle *h = nullptr;
    int nsteps = 0, every = 0, nseg = 0, S = 0;
    unsigned long long k0 = 0, k_final = 0;
    std::vector<unsigned long long> kseg;  // substep counter at each checkpoint (host copies for async uploads)
    float *x0 = nullptr, *v0 = nullptr;    // initial state, AoS [N][3]
    float *ckpt = nullptr;                 // nseg x 6 planes
    float *seg = nullptr;                  // 2 sets x (every*substeps+1) slots x 19 planes (x, v, v*, response data)
    uint32_t *cbits = nullptr;             // every*substeps+1 slots x stride/32 hit-bit words
    size_t seg_slots = 0;                  // slots per recompute set (two sets: seg and cbits hold both)
    cudaStream_t side = nullptr;           // the reverse chain of the backward pass
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
    float *lam = nullptr;                  // lx, lv, lS, lvp, lF (two buffers): 18 planes
    double *gslot = nullptr;               // gks, gkd: 12 planes (double sums over substeps)
    float *final_state = nullptr;          // 6 planes
    int *map = nullptr;                    // canonical spring -> slot
    bool forward_done = false;
    // the forward chain and the reverse pass as CUDA graphs (captured on first
    // use; rebuilt when the cloth's kernel parameters change)
    cudaGraphExec_t fwd_graph = nullptr, bwd_graph = nullptr;
    unsigned long long fwd_gen = 0, bwd_gen = 0;
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

int seg_steps(const ClothRollout *ro, int g) { return (g == ro->nseg - 1) ? ro->nsteps - g * ro->every : ro->every; }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int blocks, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)ADJ_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

cudaError_t copy_planes(const float *src, float *dst, long long nfloats, cudaStream_t s)
{
    const long long n4 = nfloats / 4;
    const long long b = (n4 + 255) / 256;
    copy_planes_kernel<<<(int)(b < 1 ? 1 : (b > 4096 ? 4096 : b)), 256, 0, s>>>((const float4 *)src, (float4 *)dst,
                                                                                  n4);
    return cudaGetLastError();
}

// The forward chain from the restored initial state: a checkpoint before
// every segment, the segment's substeps (the cloth's own launches), and a
// copy of the final state.
cudaError_t enqueue_forward(ClothRollout *ro, cudaStream_t s)
{
    ClothHandle *h = ro->h;
    const long long st = h->stride;
    cudaError_t e = cudaSuccess;
    for (int g = 0; g < ro->nseg && e == cudaSuccess; g++) {
        e = copy_planes(cur_state(h, ro->kseg[g]), ro->ckpt + (size_t)g * 6 * st, 6 * st, s);
        const int n = seg_steps(ro, g) * h->desc.substeps;
        for (int q = 0; q < n && e == cudaSuccess; q++) e = launch_substep(h->params, s);
    }
    if (e == cudaSuccess) e = copy_planes(cur_state(h, ro->k_final), ro->final_state, 6 * st, s);
    return e;
}

// Slot j of recompute set b (segments alternate between the two sets).
float *seg_slot(const ClothRollout *ro, int b, int j)
{
    return ro->seg + ((size_t)b * ro->seg_slots + (size_t)j) * SLOT_PLANES * ro->h->stride;
}
uint32_t *seg_bits(const ClothRollout *ro, int b, int j)
{
    return ro->cbits + ((size_t)b * ro->seg_slots + (size_t)j) * (size_t)(ro->h->stride / 32);
}

// Recompute of segment g from its checkpoint into slot set g & 1, with the
// substep kernels redirected: substep j reads slot j (the checkpoint for
// j = 0) and writes slot j + 1, its post-integration velocity and, for the
// nodes that hit, the response data into slot j; every substep's start state
// stays in place without copies and the cloth's state buffers are not
// touched.
cudaError_t recompute_segment(ClothRollout *ro, int g, cudaStream_t s)
{
    ClothHandle *h = ro->h;
    const long long st = h->stride;
    const int b = g & 1, nsub = seg_steps(ro, g) * h->desc.substeps;
    const unsigned long long kg = ro->kseg[g];
    const float *ck = ro->ckpt + (size_t)g * 6 * st;
    const StepParams &p = h->params;
    const long long nwords = (long long)nsub * (st / 32);
    const int zb = nblk(nwords, 256);
    segment_begin_kernel<<<zb < 1 ? 1 : (zb > 1024 ? 1024 : zb), 256, 0, s>>>(h->ctrl, kg, seg_bits(ro, b, 0),
                                                                               nwords);
    cudaError_t e = cudaGetLastError();
    for (int j = 0; j < nsub && e == cudaSuccess; j++) {
        StepParams q = p;
        float *in = j == 0 ? const_cast<float *>(ck) : seg_slot(ro, b, j);
        float *out = seg_slot(ro, b, j + 1);
        // the kernels read (k odd ? state1 : state0) and write the other
        if ((kg + (unsigned long long)j) & 1ull) {
            q.state1 = in;
            q.state0 = out;
        } else {
            q.state0 = in;
            q.state1 = out;
        }
        q.vstar = seg_slot(ro, b, j) + 6 * st;
        if (p.has_mesh) {
            q.cdata = seg_slot(ro, b, j) + 9 * st;
            q.cbits = seg_bits(ro, b, j);
        }
        e = launch_substep(q, s);
    }
    return e;
}

// Reverse of segment g over slot set g & 1, the force adjoints of
// consecutive substeps alternating between two buffers.
cudaError_t reverse_segment(ClothRollout *ro, int g, cudaStream_t s)
{
    ClothHandle *h = ro->h;
    const long long st = h->stride;
    const int b = g & 1, nsub = seg_steps(ro, g) * h->desc.substeps;
    const float *ck = ro->ckpt + (size_t)g * 6 * st;
    float *lF2[2] = {ro->lam + 12 * st, ro->lam + 15 * st};
    const int blocks = nblk((long long)h->desc.ny * h->pitch * ADJ_LANES, ADJ_THREADS);
    const StepParams &p = h->params;
    auto xstart = [&](int j) { return j == 0 ? ck : (const float *)seg_slot(ro, b, j); };
    AdjArgs a{};
    a.lS = ro->lam + 6 * st;
    a.lvp = ro->lam + 9 * st;
    a.lx = ro->lam;
    a.lv = ro->lam + 3 * st;
    a.gks = ro->gslot;
    a.gkd = ro->gslot + 6 * st;
    cudaError_t e = cudaSuccess;
    for (int j = nsub; j >= 0 && e == cudaSuccess; j--) {
        // spring part: substep j (j < nsub); contact part: substep j - 1 (j > 0)
        if (j < nsub) {
            a.xs_s = xstart(j);
            a.lF_s = lF2[j & 1];
        }
        if (j > 0) {
            a.xs_c = xstart(j - 1);
            a.vs_c = seg_slot(ro, b, j - 1) + 6 * st;
            a.cd_c = seg_slot(ro, b, j - 1) + 9 * st;
            a.cb_c = p.has_mesh ? seg_bits(ro, b, j - 1) : nullptr;
            a.lF_c = lF2[(j - 1) & 1];
        }
        if (j == nsub)
            e = launch_pdl(adj_kernel<false, true>, blocks, s, p, a);
        else if (j > 0)
            e = launch_pdl(adj_kernel<true, true>, blocks, s, p, a);
        else
            e = launch_pdl(adj_kernel<true, false>, blocks, s, p, a);
    }
    return e;
}

// The reverse pass over all segments, last first, as two chains: the
// recomputes on s and the reverse launches on the rollout's side stream.
// The reverse of segment g waits for its recompute; the recompute of
// segment g - 1 runs meanwhile (into the other slot set) and the one of
// g - 2 waits until the reverse of g has released its set.  Both chains are
// latency-bound and occupy few SMs, so they overlap.
cudaError_t enqueue_backward(ClothRollout *ro, cudaStream_t s)
{
    cudaStream_t v = ro->side;
    cudaError_t e = cudaEventRecord(ro->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(v, ro->ev_fork, 0);
    if (e != cudaSuccess) return e;
    for (int g = ro->nseg - 1; g >= 0 && e == cudaSuccess; g--) {
        if (g + 2 < ro->nseg) e = cudaStreamWaitEvent(s, ro->ev_rev[g & 1], 0);
        if (e == cudaSuccess) e = recompute_segment(ro, g, s);
        if (e == cudaSuccess) e = cudaEventRecord(ro->ev_rec[g & 1], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v, ro->ev_rec[g & 1], 0);
        if (e == cudaSuccess) e = reverse_segment(ro, g, v);
        if (e == cudaSuccess) e = cudaEventRecord(ro->ev_rev[g & 1], v);
    }
    // join the side stream back (also after an error, so that a capture ends)
    const cudaError_t j1 = cudaEventRecord(ro->ev_join, v);
    const cudaError_t j2 = j1 == cudaSuccess ? cudaStreamWaitEvent(s, ro->ev_join, 0) : j1;
    return e != cudaSuccess ? e : j2;
}

// Captures body(stream) on the cloth's capture stream into *exec.
template <typename F>
cudaError_t capture_graph(ClothHandle *h, cudaGraphExec_t *exec, F &&body)
{
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = body(h->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Runs the forward chain or the reverse pass on s, through a cached graph
// unless the cloth was created with CLOTH_FLAG_NO_GRAPH.
cudaError_t run_pass(ClothRollout *ro, bool backward, cudaStream_t s)
{
    ClothHandle *h = ro->h;
    auto body = [ro, backward](cudaStream_t cs) {
        return backward ? enqueue_backward(ro, cs) : enqueue_forward(ro, cs);
    };
    if (h->desc.flags & CLOTH_FLAG_NO_GRAPH) return body(s);
    cudaGraphExec_t &gx = backward ? ro->bwd_graph : ro->fwd_graph;
    unsigned long long &gen = backward ? ro->bwd_gen : ro->fwd_gen;
    if (gx && gen != h->params_gen) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
    }
    if (!gx) {
        const cudaError_t e = capture_graph(h, &gx, body);
        if (e != cudaSuccess) {
            gx = nullptr;
            return e;
        }
        gen = h->params_gen;
    }
    return cudaGraphLaunch(gx, s);
}

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
        for (int g = 0; g <= ro->nseg; g++)
            ro->kseg[g] = ro->k0 + (unsigned long long)g * ro->every * d.substeps;
        ro->k_final = ro->k0 + (unsigned long long)nsteps * d.substeps;
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
    const size_t seg_sub = (size_t)ro->every * d.substeps + 1;
    ro->seg_slots = seg_sub;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ro->side, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&ro->ev_fork, &ro->ev_join, &ro->ev_rec[0], &ro->ev_rec[1], &ro->ev_rev[0], &ro->ev_rev[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&ro->x0, sizeof(float) * 3 * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc(&ro->v0, sizeof(float) * 3 * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc(&ro->ckpt, sizeof(float) * 6 * (size_t)st * (size_t)ro->nseg);
    if (e == cudaSuccess) e = cudaMalloc(&ro->seg, sizeof(float) * SLOT_PLANES * (size_t)st * 2 * seg_sub);
    // the padding columns of the recompute slots match the cloth's (zero) ones
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ro->seg, 0, sizeof(float) * SLOT_PLANES * (size_t)st * 2 * seg_sub, h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&ro->cbits, sizeof(uint32_t) * (size_t)(st / 32) * 2 * seg_sub);
    if (e == cudaSuccess) e = cudaMalloc(&ro->lam, sizeof(float) * 18 * (size_t)st);
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
            for (cudaGraphExec_t &g : h->graph) {
                if (g) cudaGraphExecDestroy(g);
                g = nullptr;
            }
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
    // a cloth of one row and one column has no springs (S = 0): nothing to scatter or gather
    if (d_ks && ro->S > 0) scatter_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(d_ks, ro->map, ro->S, h->ks_slot);
    if (d_kd && ro->S > 0) scatter_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(d_kd, ro->map, ro->S, h->kd_slot);
    RTRY(h, cudaGetLastError(), "constants scatter");
    ro->kseg[0] = ro->k0;
    RTRY(h, cudaMemcpyAsync(&h->ctrl->k, &ro->kseg[0], sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
         "set substep counter");
    RTRY(h, launch_aos_to_soa(ro->x0, d_v0 ? d_v0 : ro->v0, h->state, h->state + 6 * st, st, h->n, h->desc.nx,
                              h->pitch, h->ctrl, s),
         "initial state");
    RTRY(h, run_pass(ro, false, s), "forward chain");
    h->substeps_done = (long long)ro->k_final;
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
    const int n = h->n, nx = h->desc.nx;
    cudaStream_t s = h->stream;
    float *lx = ro->lam, *lv = ro->lam + 3 * st;
    RTRY(h, cudaMemsetAsync(ro->lam, 0, sizeof(float) * 18 * st, s), "clear adjoints");
    RTRY(h, cudaMemsetAsync(ro->gslot, 0, sizeof(double) * 12 * st, s), "clear gradients");
    aos_planes_kernel<<<nblk(n, 256), 256, 0, s>>>(d_gpos, n, nx, h->pitch, st, lx);
    aos_planes_kernel<<<nblk(n, 256), 256, 0, s>>>(d_gvel, n, nx, h->pitch, st, lv);
    RTRY(h, cudaGetLastError(), "load output adjoints");
    RTRY(h, run_pass(ro, true, s), "reverse pass");
    if (d_gv0) planes_aos_kernel<<<nblk(n, 256), 256, 0, s>>>(lv, n, nx, h->pitch, st, d_gv0);
    if (d_gks && ro->S > 0) gather_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(ro->gslot, ro->map, ro->S, d_gks);
    if (d_gkd && ro->S > 0)
        gather_kernel<<<nblk(ro->S, 256), 256, 0, s>>>(ro->gslot + 6 * st, ro->map, ro->S, d_gkd);
    RTRY(h, cudaGetLastError(), "gradient outputs");
    // leave the cloth in its final forward state
    RTRY(h, cudaMemcpyAsync(&h->ctrl->k, &ro->k_final, sizeof(unsigned long long), cudaMemcpyHostToDevice, s),
         "set substep counter");
    RTRY(h, copy_planes(ro->final_state, cur_state(h, ro->k_final), 6 * st, s), "restore final state");
    return CLOTH_OK;
}

void cloth_rollout_destroy(ClothRollout *ro)
{
    if (!ro) return;
    if (ro->h) cudaStreamSynchronize(ro->h->stream);
    if (ro->side) cudaStreamSynchronize(ro->side);
    if (ro->fwd_graph) cudaGraphExecDestroy(ro->fwd_graph);
    if (ro->bwd_graph) cudaGraphExecDestroy(ro->bwd_graph);
    cudaFree(ro->x0);
    cudaFree(ro->v0);
    cudaFree(ro->ckpt);
    cudaFree(ro->seg);
    cudaFree(ro->cbits);
    if (ro->side) cudaStreamDestroy(ro->side);
    for (cudaEvent_t ev : {ro->ev_fork, ro->ev_join, ro->ev_rec[0], ro->ev_rec[1], ro->ev_rev[0], ro->ev_rev[1]})
        if (ev) cudaEventDestroy(ev);
    cudaFree(ro->lam);
    cudaFree(ro->gslot);
    cudaFree(ro->final_state);
    cudaFree(ro->map);
    cudaGetLastError();
    delete ro;
}

}  // extern "C"
