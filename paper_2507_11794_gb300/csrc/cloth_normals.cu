// Per-vertex normals of the cloth grid: the normal update that precedes
// rendering at the end of a frame (Section 3).  Each grid quad is split along
// its (r,c)-(r+1,c+1) diagonal into the triangles (r,c)-(r+1,c)-(r+1,c+1) and
// (r,c)-(r+1,c+1)-(r,c+1); a vertex normal is the normalised sum of the
// unnormalised face normals (e1 x e2) of the up to six triangles containing
// the vertex, and zero where that sum is zero.  Every face is computed once,
// and each vertex sums its faces in a fixed order (no atomics).
#include "cloth_internal.h"

namespace {

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// The kernel walks down the grid.  A warp owns a strip of 32 columns (the
// 30 of lanes 1..30 are its outputs; neighbouring strips overlap by two
// columns) and R consecutive rows.  Lane l at column c computes the two face
// normals of quad (r, c) (corners (r,c), (r,c+1), (r+1,c), (r+1,c+1)) once
// per row from its own column and lane l+1's (a shuffle); vertex (r, c)
// then takes the faces it lies in from its own quads (r, c) and (r-1, c)
// (the latter kept from the previous row) and from lane l-1's quads (r, c-1)
// and (r-1, c-1).  Each face is the triangle's (b - a) x (c - a) from its
// first corner in the order above, and a vertex adds its faces in the
// order: quad (r,c) both, quad (r-1,c) first, quad (r,c-1) second, quad
// (r-1,c-1) both.  Rows and columns outside the grid are loaded clamped into
// it and their quads are left out.  Positions are read once per strip row
// (plus one halo row above and one below).
constexpr int NW_OUT = 30;   // output columns of a warp (lanes 1..30)
constexpr int NW_WARPS = 4;  // warps per CTA

// face normal of the triangle (a, b, c): (b - a) x (c - a)
__device__ __forceinline__ V3 face(V3 a, V3 b, V3 c) { return cross(sub(b, a), sub(c, a)); }
__device__ __forceinline__ void acc(V3 &n, V3 f)
{
    n.x += f.x;
    n.y += f.y;
    n.z += f.z;
}
__device__ __forceinline__ V3 shfl_down3(V3 a)
{
    return {__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1),
            __shfl_down_sync(0xffffffffu, a.z, 1)};
}
__device__ __forceinline__ V3 shfl_up3(V3 a)
{
    return {__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1),
            __shfl_up_sync(0xffffffffu, a.z, 1)};
}

template <int R>
__global__ void __launch_bounds__(32 * NW_WARPS) normals_kernel(const float *__restrict__ px,
                                                                const float *__restrict__ py,
                                                                const float *__restrict__ pz, int nx, int ny,
                                                                int pitch, int strips_x, int strips_y,
                                                                float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * NW_WARPS + (threadIdx.x >> 5);
    if (w >= (long long)strips_x * strips_y) return;  // whole warps only
    const int sx = (int)(w % strips_x), sy = (int)(w / strips_x);
    const int c = sx * NW_OUT - 1 + lane;
    const int cm = min(max(c, 0), nx - 1);
    const int r0 = sy * R;
    // every row the strip needs (r0 - 1 .. r0 + R) is loaded up front, each
    // clamped into the grid, so the loads overlap
    V3 P[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; k++) {
        const int rr = min(max(r0 - 1 + k, 0), ny - 1);
        const unsigned o = (unsigned)rr * (unsigned)pitch + (unsigned)cm;
        P[k] = V3{__ldg(px + o), __ldg(py + o), __ldg(pz + o)};
    }
    // quads of column c (own) and c - 1 (left) exist column-wise
    const bool qc = c >= 0 && c + 1 < nx, ql = c >= 1 && c < nx;
    const bool out_ok = lane >= 1 && lane <= NW_OUT && c < nx;

    // quads (r0 - 1, c) and (r0 - 1, c - 1), for row r0's vertices
    V3 bv = shfl_down3(P[1]);  // (r0, c + 1)
    const V3 bu = shfl_down3(P[0]);
    V3 u1 = face(P[0], P[1], bv), u2 = face(P[0], bv, bu);
    bool vu = qc && r0 >= 1;
    V3 lu1 = shfl_up3(u1), lu2 = shfl_up3(u2);
    bool vlu = ql && r0 >= 1;
#pragma unroll
    for (int k = 1; k <= R; k++) {
        const int r = r0 - 1 + k;  // P[k] is row r, P[k + 1] row r + 1
        const V3 bd = shfl_down3(P[k + 1]);  // (r + 1, c + 1)
        const V3 q1 = face(P[k], P[k + 1], bd), q2 = face(P[k], bd, bv);
        const bool vq = qc && r + 1 < ny, vl = ql && r + 1 < ny;
        const V3 l1 = shfl_up3(q1), l2 = shfl_up3(q2);
        V3 n = {0.0f, 0.0f, 0.0f};
        if (vq) {
            acc(n, q1);
            acc(n, q2);
        }
        if (vu) acc(n, u1);
        if (vl) acc(n, l2);
        if (vlu) {
            acc(n, lu1);
            acc(n, lu2);
        }
        if (out_ok && r < ny) {
            const float s2 = n.x * n.x + n.y * n.y + n.z * n.z;
            const float s = s2 > 0.0f ? rsqrtf(s2) : 0.0f;  // within 2 ulp of 1 / sqrt
            float *o = out + 3 * ((long long)r * nx + c);
            o[0] = n.x * s;
            o[1] = n.y * s;
            o[2] = n.z * s;
        }
        u1 = q1;
        u2 = q2;
        vu = vq;
        lu1 = l1;
        lu2 = l2;
        vlu = vl;
        bv = bd;
    }
}

// rows per warp: 5 at 800 x 800 gives 4,320 warps, about 28 per SM in one wave
#ifndef CLOTH_NORMALS_ROWS
#define CLOTH_NORMALS_ROWS 5
#endif
constexpr int NW_ROWS = CLOTH_NORMALS_ROWS;

}  // namespace

cudaError_t launch_normals(const float *state, long long stride, int nx, int ny, int pitch, float *out, int /*sms*/,
                           cudaStream_t s)
{
    const long long strips_x = (nx + NW_OUT - 1) / NW_OUT;
    const long long strips_y = (ny + NW_ROWS - 1) / NW_ROWS;
    const long long blocks = (strips_x * strips_y + NW_WARPS - 1) / NW_WARPS;
    normals_kernel<NW_ROWS><<<(unsigned)blocks, 32 * NW_WARPS, 0, s>>>(state, state + stride, state + 2 * stride, nx,
                                                                       ny, pitch, (int)strips_x, (int)strips_y, out);
    return cudaGetLastError();
}
