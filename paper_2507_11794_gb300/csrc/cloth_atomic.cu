// Spring forces as Algorithm 1 prints them, for the A/B against the fused
// column walk: one thread per spring adds F to its first node and -F to its
// second with FP32 atomic adds into a per-node force buffer; one thread per
// node then integrates (symplectic Euler with pins, gravity and wind,
// Section 3), zeroes its force accumulator for the next substep (as
// Algorithm 2 resets its buffers), and lists the nodes whose path box reaches
// the surface model's grid for the collision kernel.
//
// The force law, the integrator and the collision phase are those of the
// default path; only the order of the force additions differs and varies
// from run to run.
#include "cloth_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SPRING_THREADS = 256;
constexpr int NODE_THREADS = 256;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Direction d of the canonical order: (0,+1) (+1,0) (+1,+1) (+1,-1) (0,+2) (+2,0),
// spring types 0 0 1 1 2 2.
__device__ __forceinline__ int dir_dr(int d) { return d == 0 || d == 4 ? 0 : (d == 5 ? 2 : 1); }
__device__ __forceinline__ int dir_dc(int d) { return d == 0 ? 1 : (d == 1 || d == 5 ? 0 : (d == 2 ? 1 : (d == 3 ? -1 : 2))); }
__device__ __forceinline__ int dir_type(int d) { return d >> 1; }

// Algorithm 1, one thread per spring slot (direction-major, so consecutive
// threads take consecutive nodes of one direction): dir = normalize(p2 - p1),
// springForce = ks (|p2 - p1| - L0), dampingForce = kd (v2.dir - v1.dir),
// F = (springForce + dampingForce) dir; F to node 1, -F to node 2.  A spring
// of length <= 1e-12 (|d|^2 <= 1e-24) contributes nothing.
__global__ void __launch_bounds__(SPRING_THREADS) spring_atomic_kernel(const __grid_constant__ StepParams p)
{
    __shared__ unsigned long long s_k;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) s_k = *(volatile unsigned long long *)&p.ctrl->k;
    __syncthreads();
    const unsigned long long k = s_k;
    const float *__restrict__ in = (k & 1ull) ? p.state1 : p.state0;
    const long long st = p.stride;
    const long long nodes = (long long)p.nx * p.ny;
    const long long total = 6 * nodes;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(t / nodes);
        const long long rem = t - (long long)d * nodes;
        const int r = (int)(rem / p.nx), c = (int)(rem - (long long)r * p.nx);
        const int r2 = r + dir_dr(d), c2 = c + dir_dc(d);
        if (r2 >= p.ny || c2 < 0 || c2 >= p.nx) continue;  // no spring in this slot
        const unsigned o1 = (unsigned)r * (unsigned)p.pitch + (unsigned)c;
        const unsigned o2 = (unsigned)r2 * (unsigned)p.pitch + (unsigned)c2;
        float ks, kd;
        if (p.ks_slot) {
            ks = __ldg(p.ks_slot + d * st + o1);
            kd = __ldg(p.kd_slot + d * st + o1);
        } else {
            ks = p.ks[dir_type(d)];
            kd = p.kd[dir_type(d)];
        }
        const float dx = __ldg(in + o2) - __ldg(in + o1);
        const float dy = __ldg(in + st + o2) - __ldg(in + st + o1);
        const float dz = __ldg(in + 2 * st + o2) - __ldg(in + 2 * st + o1);
        const float l2 = dx * dx + dy * dy + dz * dz;
        if (!(l2 > 1e-24f)) continue;
        const float l = sqrtf(l2);
        const float ux = dx / l, uy = dy / l, uz = dz / l;
        const float springForce = ks * (l - p.L0[d]);
        const float v1 = __ldg(in + 3 * st + o1) * ux + __ldg(in + 4 * st + o1) * uy + __ldg(in + 5 * st + o1) * uz;
        const float v2 = __ldg(in + 3 * st + o2) * ux + __ldg(in + 4 * st + o2) * uy + __ldg(in + 5 * st + o2) * uz;
        const float dampingForce = kd * (v2 - v1);
        const float f = springForce + dampingForce;
        atomicAdd(p.force + o1, make_float4(f * ux, f * uy, f * uz, 0.0f));
        atomicAdd(p.force + o2, make_float4(-f * ux, -f * uy, -f * uz, 0.0f));
    }
}

// One thread per node: integrate, reset the accumulator, mark for collision.
template <bool MESH>
__global__ void __launch_bounds__(NODE_THREADS) node_integrate_kernel(const __grid_constant__ StepParams p)
{
    __shared__ unsigned long long s_k;
    __shared__ float s_sinW, s_cosW;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) {
        const unsigned long long k = *(volatile unsigned long long *)&p.ctrl->k;
        s_k = k;
        float sw = 0.0f, cw = 1.0f;
        if (p.has_wind) sincosf(wind_base(p.w_turn_step, p.w_turn0, k), &sw, &cw);
        s_sinW = sw;
        s_cosW = cw;
    }
    __syncthreads();
    const unsigned long long k = s_k;
    const float *__restrict__ in = (k & 1ull) ? p.state1 : p.state0;
    float *__restrict__ out = (k & 1ull) ? p.state0 : p.state1;
    const long long st = p.stride;
    const long long nodes = (long long)p.nx * p.ny;
    const int lane = threadIdx.x & 31;
    float fsum = 0.0f;
    // the block's base index is uniform, so every lane of a warp runs the same
    // number of iterations (the list append below is warp-collective)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nodes; base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool valid = i < nodes;
        bool need = false;
        unsigned o = 0u;
        if (valid) {
            const int r = (int)(i / p.nx), c = (int)(i - (long long)(i / p.nx) * p.nx);
            o = (unsigned)r * (unsigned)p.pitch + (unsigned)c;
            const float4 F = p.force[o];
            p.force[o] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const float px = __ldg(in + o), py = __ldg(in + st + o), pz = __ldg(in + 2 * st + o);
            const float vx = __ldg(in + 3 * st + o), vy = __ldg(in + 4 * st + o), vz = __ldg(in + 5 * st + o);
            bool pinned = false;
            if (p.pin_bits) pinned = (__ldg(p.pin_bits + (o >> 5)) >> (o & 31u)) & 1u;
            float ax = fmaf(F.x, p.inv_mass, p.g[0]);
            float ay = fmaf(F.y, p.inv_mass, p.g[1]);
            float az = fmaf(F.z, p.inv_mass, p.g[2]);
            if (p.has_wind) {
                // sin(a + b) = sin(a) cos(b) + cos(a) sin(b), a = base + alpha_r, b = beta_c
                const float2 tr = __ldg(p.wind_rows + r), tc = __ldg(p.wind_cols + c);
                const float sinR = s_sinW * tr.y + s_cosW * tr.x;
                const float cosR = s_cosW * tr.y - s_sinW * tr.x;
                const float w = p.w_amp * (cosR * tc.x + sinR * tc.y);
                ax = fmaf(w, p.w_dir[0], ax);
                ay = fmaf(w, p.w_dir[1], ay);
                az = fmaf(w, p.w_dir[2], az);
            }
            float wx = fmaf(p.dt, ax, vx), wy = fmaf(p.dt, ay, vy), wz = fmaf(p.dt, az, vz);
            float xx = fmaf(p.dt, wx, px), xy = fmaf(p.dt, wy, py), xz = fmaf(p.dt, wz, pz);
            if (pinned) {  // kinematic: x += dt u, v = u (u = 0: fixed)
                xx = fmaf(p.dt, p.pin_vel[0], px); xy = fmaf(p.dt, p.pin_vel[1], py); xz = fmaf(p.dt, p.pin_vel[2], pz);
                wx = p.pin_vel[0]; wy = p.pin_vel[1]; wz = p.pin_vel[2];
            }
            if (MESH)
                need = !pinned && fmaxf(px, xx) >= p.mlo[0] && fminf(px, xx) <= p.mhi[0] &&
                       fmaxf(py, xy) >= p.mlo[1] && fminf(py, xy) <= p.mhi[1] && fmaxf(pz, xz) >= p.mlo[2] &&
                       fminf(pz, xz) <= p.mhi[2];
            if (p.vstar) {
                p.vstar[o] = wx;
                p.vstar[st + o] = wy;
                p.vstar[2 * st + o] = wz;
            }
            out[o] = xx;
            out[st + o] = xy;
            out[2 * st + o] = xz;
            out[3 * st + o] = wx;
            out[4 * st + o] = wy;
            out[5 * st + o] = wz;
            fsum += ((xx + xy) + (xz + wx)) + (wy + wz);
        }
        if (MESH) {
            const unsigned m = __ballot_sync(FULL, need);
            if (m) {
                unsigned w0 = 0;
                if (lane == 0) w0 = atomicAdd(p.coll_count, (unsigned)__popc(m));
                w0 = __shfl_sync(FULL, w0, 0);
                if (need) p.coll_list[w0 + __popc(m & ((1u << lane) - 1u))] = (int)o;
            }
        }
    }
    if (__any_sync(FULL, !isfinite(fsum)) && lane == 0) atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    if (MESH) return;  // the collision kernel finishes the substep
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&p.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            p.ctrl->blocks_done = 0;
            p.ctrl->k = k + 1;
        }
    }
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int blocks, int threads, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

int grid_for(long long work, int threads, int sms)
{
    const long long b = (work + threads - 1) / threads;
    const long long cap = (long long)sms * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_atomic_forces_and_integrate(const StepParams &p, cudaStream_t s)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long nodes = (long long)p.nx * p.ny;
    cudaError_t e = launch_pdl(spring_atomic_kernel, grid_for(6 * nodes, SPRING_THREADS, sms), SPRING_THREADS, s, p);
    if (e != cudaSuccess) return e;
    const int nb = grid_for(nodes, NODE_THREADS, sms);
    return p.has_mesh ? launch_pdl(node_integrate_kernel<true>, nb, NODE_THREADS, s, p)
                      : launch_pdl(node_integrate_kernel<false>, nb, NODE_THREADS, s, p);
}
