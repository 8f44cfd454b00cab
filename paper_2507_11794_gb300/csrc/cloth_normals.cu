// Per-vertex normals of the cloth grid: the normal update that precedes
// rendering at the end of a frame (Section 3).  Each grid quad is split along
// its (r,c)-(r+1,c+1) diagonal into the triangles (r,c)-(r+1,c)-(r+1,c+1) and
// (r,c)-(r+1,c+1)-(r,c+1); a vertex normal is the normalised sum of the
// unnormalised face normals (e1 x e2) of the up to six triangles containing
// the vertex, and zero where that sum is zero.  One thread per node gathers
// its triangles (no atomics, fixed order).
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
// face normal of the triangle (a, b, c): (b - a) x (c - a)
__device__ __forceinline__ void add_face(V3 &n, V3 a, V3 b, V3 c)
{
    const V3 f = cross(sub(b, a), sub(c, a));
    n.x += f.x;
    n.y += f.y;
    n.z += f.z;
}

// Block (x, y): columns [NB_COLS x, NB_COLS (x+1)) of rows y, y + gridDim.y, ...,
// one node per thread.
constexpr int NB_COLS = 128;

__global__ void __launch_bounds__(NB_COLS) normals_kernel(const float *__restrict__ px, const float *__restrict__ py,
                                                          const float *__restrict__ pz, int nx, int ny, int pitch,
                                                          float *__restrict__ out)
{
    const int c = blockIdx.x * NB_COLS + threadIdx.x;
    if (c >= nx) return;
    for (int r = blockIdx.y; r < ny; r += gridDim.y) {
        auto P = [&](int rr, int cc) {
            const unsigned o = (unsigned)rr * (unsigned)pitch + (unsigned)cc;
            return V3{__ldg(px + o), __ldg(py + o), __ldg(pz + o)};
        };
        const bool up = r >= 1, down = r + 1 < ny, left = c >= 1, right = c + 1 < nx;
        // all seven points are loaded unconditionally (clamped into the grid)
        // so their loads overlap; the branches below only select the faces
        const int ru = up ? r - 1 : r, rd = down ? r + 1 : r, cl = left ? c - 1 : c, cr = right ? c + 1 : c;
        const V3 v = P(r, c), d = P(rd, c), e = P(rd, cr), b = P(r, cr), u = P(ru, c), l = P(r, cl),
                 a = P(ru, cl);
        V3 n = {0.0f, 0.0f, 0.0f};
        if (down && right) {  // quad (r, c): both triangles
            add_face(n, v, d, e);
            add_face(n, v, e, b);
        }
        if (up && right) add_face(n, u, v, b);    // quad (r-1, c), first triangle
        if (down && left) add_face(n, l, d, v);   // quad (r, c-1), second triangle
        if (up && left) {                         // quad (r-1, c-1): both
            add_face(n, a, l, v);
            add_face(n, a, v, u);
        }
        const float l2 = n.x * n.x + n.y * n.y + n.z * n.z;
        const float s = l2 > 0.0f ? 1.0f / sqrtf(l2) : 0.0f;
        float *o = out + 3 * ((long long)r * nx + c);
        o[0] = n.x * s;
        o[1] = n.y * s;
        o[2] = n.z * s;
    }
}

}  // namespace

cudaError_t launch_normals(const float *state, long long stride, int nx, int ny, int pitch, float *out, int /*sms*/,
                           cudaStream_t s)
{
    const dim3 grid((unsigned)((nx + NB_COLS - 1) / NB_COLS), (unsigned)(ny < 65535 ? ny : 65535));
    normals_kernel<<<grid, NB_COLS, 0, s>>>(state, state + stride, state + 2 * stride, nx, ny, pitch, out);
    return cudaGetLastError();
}
