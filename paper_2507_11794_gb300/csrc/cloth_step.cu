// One substep of the mass-spring cloth, fused into a single kernel:
//   spring + damping forces (Algorithm 1's force law, gathered per node),
//   symplectic Euler with gravity, wind and pins (Section 3),
//   uniform-grid broad phase + extended Moller-Trumbore narrow phase on the
//   node's substep path (Section 3) and the averaged response of Algorithm 2.
//
// Layout: six SoA float planes (px py pz vx vy vz) per ping-pong buffer; the
// launch reads buffer k&1 and writes the other, k = the device substep counter.
// Each CTA stages a TX x TY node tile plus a two-node halo (bend springs reach
// two nodes) of all six planes in shared memory, then each thread gathers the
// twelve springs of its nodes from shared memory: no atomics, fixed summation
// order, so results are bitwise reproducible run to run.
#include "cloth_internal.h"

namespace {

constexpr int TX = 32;           // tile columns (one warp)
constexpr int TY = 16;           // tile rows
constexpr int BY = 8;            // thread rows per CTA; each thread owns TY/BY nodes
constexpr int HALO = 2;
constexpr int SX = TX + 2 * HALO;
constexpr int SY = TY + 2 * HALO;
constexpr int NTHREADS = TX * BY;

__device__ __forceinline__ void spring_add(float pix, float piy, float piz, float vix, float viy, float viz,
                                           float pjx, float pjy, float pjz, float vjx, float vjy, float vjz,
                                           float ks, float kd, float L0, float &fx, float &fy, float &fz)
{
    // Hooke's law plus damping along the spring (Algorithm 1), seen from node i:
    // d = p_j - p_i, F_i += (ks (|d| - L0) + kd (v_j - v_i).d^) d^.
    float dx = pjx - pix, dy = pjy - piy, dz = pjz - piz;
    float l2 = dx * dx + dy * dy + dz * dz;
    if (l2 > 1e-24f) {
        float il = rsqrtf(l2);
        float l = l2 * il;
        float ux = dx * il, uy = dy * il, uz = dz * il;
        float dvn = (vjx - vix) * ux + (vjy - viy) * uy + (vjz - viz) * uz;
        float f = ks * (l - L0) + kd * dvn;
        fx += f * ux;
        fy += f * uy;
        fz += f * uz;
    }
}

template <bool MESH, bool PER_SPRING>
__global__ void __launch_bounds__(NTHREADS) substep_kernel(const StepParams p)
{
    constexpr int DR[CLOTH_NDIR] = {0, 1, 1, 1, 0, 2};
    constexpr int DC[CLOTH_NDIR] = {1, 0, 1, -1, 2, 0};
    constexpr int TYPE[CLOTH_NDIR] = {0, 0, 1, 1, 2, 2};

    __shared__ float sm[6][SY][SX];
    __shared__ unsigned long long s_k;
    __shared__ float s_wbase;

    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        unsigned long long k = *(volatile unsigned long long *)&p.ctrl->k;
        s_k = k;
        float wb = 0.0f;
        if (p.has_wind) {
            // omega*k + phase0 reduced mod 2*pi in double, once per CTA
            double ph = fmod(p.w_omega * (double)k + p.w_phase0, 6.283185307179586);
            wb = (float)ph;
        }
        s_wbase = wb;
    }
    __syncthreads();
    const unsigned long long k = s_k;
    const float *__restrict__ in = (k & 1ull) ? p.state1 : p.state0;
    float *__restrict__ out = (k & 1ull) ? p.state0 : p.state1;
    const long long st = p.stride;
    const int c0 = blockIdx.x * TX, r0 = blockIdx.y * TY;

    for (int idx = tid; idx < SX * SY; idx += NTHREADS) {
        int ly = idx / SX, lx = idx - ly * SX;
        int r = r0 - HALO + ly, c = c0 - HALO + lx;
        bool ok = (r >= 0) && (r < p.ny) && (c >= 0) && (c < p.nx);
        long long g = (long long)r * p.nx + c;
#pragma unroll
        for (int q = 0; q < 6; q++) sm[q][ly][lx] = ok ? __ldg(in + q * st + g) : 0.0f;
    }
    __syncthreads();

    bool bad = false;
#pragma unroll 1
    for (int jrow = 0; jrow < TY / BY; jrow++) {
        const int ly = threadIdx.y + jrow * BY, lx = threadIdx.x;
        const int r = r0 + ly, c = c0 + lx;
        if (r >= p.ny || c >= p.nx) continue;
        const int i = r * p.nx + c;
        const int sy = ly + HALO, sx = lx + HALO;
        const float pix = sm[0][sy][sx], piy = sm[1][sy][sx], piz = sm[2][sy][sx];
        const float vix = sm[3][sy][sx], viy = sm[4][sy][sx], viz = sm[5][sy][sx];

        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
        for (int d = 0; d < CLOTH_NDIR; d++) {
            // spring owned by this node, towards (+DR, +DC)
            {
                const int rr = r + DR[d], cc = c + DC[d];
                if (rr < p.ny && cc >= 0 && cc < p.nx) {
                    const float ks = PER_SPRING ? __ldg(p.ks_slot + d * st + i) : p.ks[TYPE[d]];
                    const float kd = PER_SPRING ? __ldg(p.kd_slot + d * st + i) : p.kd[TYPE[d]];
                    const int yy = sy + DR[d], xx = sx + DC[d];
                    spring_add(pix, piy, piz, vix, viy, viz, sm[0][yy][xx], sm[1][yy][xx], sm[2][yy][xx],
                               sm[3][yy][xx], sm[4][yy][xx], sm[5][yy][xx], ks, kd, p.L0[d], fx, fy, fz);
                }
            }
            // spring owned by the node at (-DR, -DC), towards this node
            {
                const int rr = r - DR[d], cc = c - DC[d];
                if (rr >= 0 && cc >= 0 && cc < p.nx) {
                    const int j = i - DR[d] * p.nx - DC[d];
                    const float ks = PER_SPRING ? __ldg(p.ks_slot + d * st + j) : p.ks[TYPE[d]];
                    const float kd = PER_SPRING ? __ldg(p.kd_slot + d * st + j) : p.kd[TYPE[d]];
                    const int yy = sy - DR[d], xx = sx - DC[d];
                    spring_add(pix, piy, piz, vix, viy, viz, sm[0][yy][xx], sm[1][yy][xx], sm[2][yy][xx],
                               sm[3][yy][xx], sm[4][yy][xx], sm[5][yy][xx], ks, kd, p.L0[d], fx, fy, fz);
                }
            }
        }

        const bool pinned = p.pin_bits && ((__ldg(p.pin_bits + (i >> 5)) >> (i & 31)) & 1u);
        float xx_, xy_, xz_, wx, wy, wz;
        if (pinned) {
            xx_ = pix; xy_ = piy; xz_ = piz;
            wx = wy = wz = 0.0f;
        } else {
            float ax = fx * p.inv_mass + p.g[0];
            float ay = fy * p.inv_mass + p.g[1];
            float az = fz * p.inv_mass + p.g[2];
            if (p.has_wind) {
                const float w = p.w_amp * sinf(s_wbase + (float)c * p.w_kc + (float)r * p.w_kr);
                ax += w * p.w_dir[0];
                ay += w * p.w_dir[1];
                az += w * p.w_dir[2];
            }
            wx = vix + p.dt * ax;
            wy = viy + p.dt * ay;
            wz = viz + p.dt * az;
            const float ex = pix + p.dt * wx, ey = piy + p.dt * wy, ez = piz + p.dt * wz;
            xx_ = ex; xy_ = ey; xz_ = ez;
            if (MESH) {
                const float dx = ex - pix, dy = ey - piy, dz = ez - piz;
                const float L = sqrtf(dx * dx + dy * dy + dz * dz);
                if (L >= p.eps) {
                    const float rx = dx / L, ry = dy / L, rz = dz / L;
                    const int lox = cell_coord(fminf(pix, ex), p.go[0], p.ginv, p.gd[0]);
                    const int hix = cell_coord(fmaxf(pix, ex), p.go[0], p.ginv, p.gd[0]);
                    const int loy = cell_coord(fminf(piy, ey), p.go[1], p.ginv, p.gd[1]);
                    const int hiy = cell_coord(fmaxf(piy, ey), p.go[1], p.ginv, p.gd[1]);
                    const int loz = cell_coord(fminf(piz, ez), p.go[2], p.ginv, p.gd[2]);
                    const int hiz = cell_coord(fmaxf(piz, ez), p.go[2], p.ginv, p.gd[2]);
                    int K = 0;
                    float acc = 0.0f;
                    for (int cz = loz; cz <= hiz; cz++)
                        for (int cy = loy; cy <= hiy; cy++)
                            for (int cx = lox; cx <= hix; cx++) {
                                const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
                                const int e0 = __ldg(p.cell_start + cell), e1 = __ldg(p.cell_start + cell + 1);
                                for (int e = e0; e < e1; e++) {
                                    const int t = __ldg(p.tri_ids + e);
                                    const float4 A = __ldg(p.tri + 3 * t);
                                    const float4 B = __ldg(p.tri + 3 * t + 1);
                                    const float4 C = __ldg(p.tri + 3 * t + 2);
                                    // a triangle listed in several cells of the box is
                                    // tested only in the first cell the two boxes share
                                    if (max(__float_as_int(A.w), lox) != cx || max(__float_as_int(B.w), loy) != cy ||
                                        max(__float_as_int(C.w), loz) != cz)
                                        continue;
                                    // extended Moller-Trumbore: S = p_i, edge direction r, length L
                                    const float hx = ry * C.z - rz * C.y;
                                    const float hy = rz * C.x - rx * C.z;
                                    const float hz = rx * C.y - ry * C.x;
                                    const float a = B.x * hx + B.y * hy + B.z * hz;
                                    if (fabsf(a) < p.eps) continue;
                                    const float f = 1.0f / a;
                                    const float sx_ = pix - A.x, sy_ = piy - A.y, sz_ = piz - A.z;
                                    const float u = f * (sx_ * hx + sy_ * hy + sz_ * hz);
                                    if (u < 0.0f || u > 1.0f) continue;
                                    const float qx = sy_ * B.z - sz_ * B.y;
                                    const float qy = sz_ * B.x - sx_ * B.z;
                                    const float qz = sx_ * B.y - sy_ * B.x;
                                    const float v = f * (rx * qx + ry * qy + rz * qz);
                                    const float th = f * (C.x * qx + C.y * qy + C.z * qz);
                                    if (v < 0.0f || u + v > 1.0f) continue;
                                    if (!(th > p.tmin && th < L)) continue;
                                    K++;
                                    acc += fmaxf(th - p.delta, 0.0f);
                                }
                            }
                    if (K > 0) {
                        const float m = acc / (float)K;
                        xx_ = pix + m * rx;
                        xy_ = piy + m * ry;
                        xz_ = piz + m * rz;
                        wx *= p.restitution;
                        wy *= p.restitution;
                        wz *= p.restitution;
                    }
                }
            }
        }
        bad |= !(isfinite(xx_) && isfinite(xy_) && isfinite(xz_) && isfinite(wx) && isfinite(wy) && isfinite(wz));
        out[0 * st + i] = xx_;
        out[1 * st + i] = xy_;
        out[2 * st + i] = xz_;
        out[3 * st + i] = wx;
        out[4 * st + i] = wy;
        out[5 * st + i] = wz;
    }

    bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (bad) atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
        // the last CTA to finish advances the substep counter for the next launch
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        const unsigned prev = atomicAdd(&p.ctrl->blocks_done, 1u);
        if (prev == total - 1) {
            p.ctrl->blocks_done = 0;
            p.ctrl->k = k + 1;
            __threadfence();
        }
    }
}

__global__ void aos_to_soa_kernel(const float *__restrict__ pos, const float *__restrict__ vel, float *state0,
                                  float *state1, long long st, int n, DevCtrl *ctrl)
{
    const unsigned long long k = *(volatile unsigned long long *)&ctrl->k;
    float *dst = (k & 1ull) ? state1 : state0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (pos) {
            dst[0 * st + i] = pos[3 * (long long)i];
            dst[1 * st + i] = pos[3 * (long long)i + 1];
            dst[2 * st + i] = pos[3 * (long long)i + 2];
        }
        if (vel) {
            dst[3 * st + i] = vel[3 * (long long)i];
            dst[4 * st + i] = vel[3 * (long long)i + 1];
            dst[5 * st + i] = vel[3 * (long long)i + 2];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->flags = 0u;
}

__global__ void soa_to_aos_kernel(const float *state0, const float *state1, long long st, int n,
                                  const DevCtrl *ctrl, float *__restrict__ pos, float *__restrict__ vel)
{
    const unsigned long long k = *(volatile const unsigned long long *)&ctrl->k;
    const float *src = (k & 1ull) ? state1 : state0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (pos) {
            pos[3 * (long long)i] = src[0 * st + i];
            pos[3 * (long long)i + 1] = src[1 * st + i];
            pos[3 * (long long)i + 2] = src[2 * st + i];
        }
        if (vel) {
            vel[3 * (long long)i] = src[3 * st + i];
            vel[3 * (long long)i + 1] = src[4 * st + i];
            vel[3 * (long long)i + 2] = src[5 * st + i];
        }
    }
}

int transfer_blocks(int n)
{
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

cudaError_t launch_substep(const StepParams &p, cudaStream_t s)
{
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
    dim3 block(TX, BY);
    const bool per = p.ks_slot != nullptr;
    if (p.has_mesh) {
        if (per) substep_kernel<true, true><<<grid, block, 0, s>>>(p);
        else substep_kernel<true, false><<<grid, block, 0, s>>>(p);
    } else {
        if (per) substep_kernel<false, true><<<grid, block, 0, s>>>(p);
        else substep_kernel<false, false><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const float *aos_pos, const float *aos_vel, float *state0, float *state1,
                              long long stride, int n, DevCtrl *ctrl, cudaStream_t s)
{
    aos_to_soa_kernel<<<transfer_blocks(n), 256, 0, s>>>(aos_pos, aos_vel, state0, state1, stride, n, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const float *state0, const float *state1, long long stride, int n,
                              const DevCtrl *ctrl, float *aos_pos, float *aos_vel, cudaStream_t s)
{
    soa_to_aos_kernel<<<transfer_blocks(n), 256, 0, s>>>(state0, state1, stride, n, ctrl, aos_pos, aos_vel);
    return cudaGetLastError();
}
