// Collision of one node's substep path with the surface model (device code
// shared by the forward and the reverse pass).
#pragma once

#include "cloth_internal.h"

// Broad + narrow phase and response of one node (scalar).  S = start, E =
// predicted end; on K > 0 hits returns true and the response position.
// GRAD also returns, for the reverse pass, K, the path length and direction,
// m = mean max(t_k - delta, 0), and over the active hits (t_k > delta) the
// sums g1 = sum n/a and g2 = sum t n/a (n = e1 x e2, a = e1.(r x e2)), the
// derivatives of t_k w.r.t. S and r.  Forward and reverse passes run this one
// function, so they see the same hits.
template <bool GRAD>
__device__ __forceinline__ bool collide_t(const StepParams &p, float sx, float sy, float sz, float ex, float ey,
                                          float ez, float &ox, float &oy, float &oz, float *g1 = nullptr,
                                          float *g2 = nullptr, float *mK = nullptr)
{
    const float dx = ex - sx, dy = ey - sy, dz = ez - sz;
    const float L = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(L >= p.eps)) return false;
    const float rx = dx / L, ry = dy / L, rz = dz / L;
    const int lox = cell_coord(fminf(sx, ex), p.go[0], p.ginv, p.gd[0]);
    const int hix = cell_coord(fmaxf(sx, ex), p.go[0], p.ginv, p.gd[0]);
    const int loy = cell_coord(fminf(sy, ey), p.go[1], p.ginv, p.gd[1]);
    const int hiy = cell_coord(fmaxf(sy, ey), p.go[1], p.ginv, p.gd[1]);
    const int loz = cell_coord(fminf(sz, ez), p.go[2], p.ginv, p.gd[2]);
    const int hiz = cell_coord(fmaxf(sz, ez), p.go[2], p.ginv, p.gd[2]);
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
                    // a triangle listed in several cells of the box is tested
                    // only in the first cell the two boxes share
                    if (max(__float_as_int(A.w), lox) != cx || max(__float_as_int(B.w), loy) != cy ||
                        max(__float_as_int(C.w), loz) != cz)
                        continue;
                    // extended Moller-Trumbore: edge S -> E, direction r, length L
                    const float hx = ry * C.z - rz * C.y;
                    const float hy = rz * C.x - rx * C.z;
                    const float hz = rx * C.y - ry * C.x;
                    const float a = B.x * hx + B.y * hy + B.z * hz;
                    if (fabsf(a) < p.eps) continue;
                    const float f = 1.0f / a;
                    const float qx0 = sx - A.x, qy0 = sy - A.y, qz0 = sz - A.z;
                    const float u = f * (qx0 * hx + qy0 * hy + qz0 * hz);
                    if (u < 0.0f || u > 1.0f) continue;
                    const float qx = qy0 * B.z - qz0 * B.y;
                    const float qy = qz0 * B.x - qx0 * B.z;
                    const float qz = qx0 * B.y - qy0 * B.x;
                    const float v = f * (rx * qx + ry * qy + rz * qz);
                    const float th = f * (C.x * qx + C.y * qy + C.z * qz);
                    if (v < 0.0f || u + v > 1.0f) continue;
                    if (!(th > p.tmin && th < L)) continue;
                    K++;
                    acc += fmaxf(th - p.delta, 0.0f);
                    if (GRAD && th - p.delta > 0.0f) {
                        const float nx = B.y * C.z - B.z * C.y, ny = B.z * C.x - B.x * C.z, nz = B.x * C.y - B.y * C.x;
                        g1[0] += nx * f; g1[1] += ny * f; g1[2] += nz * f;
                        g2[0] += th * nx * f; g2[1] += th * ny * f; g2[2] += th * nz * f;
                    }
                }
            }
    if (K == 0) return false;
    const float m = acc / (float)K;
    if (GRAD) {
        mK[0] = m;
        mK[1] = (float)K;
        mK[2] = rx; mK[3] = ry; mK[4] = rz;
    }
    ox = sx + m * rx;
    oy = sy + m * ry;
    oz = sz + m * rz;
    return true;
}

// One warp's strip: columns [60 sx - 2, 60 sx + 62) walked down rows
// [r0 - 2, r0 + rows_per_warp); writes rows [r0, r1) of the output state and,
// with a surface model, appends the nodes that need the collision kernel.

__device__ __forceinline__ bool collide(const StepParams &p, float sx, float sy, float sz, float ex, float ey, float ez,
                                        float &ox, float &oy, float &oz)
{
    return collide_t<false>(p, sx, sy, sz, ex, ey, ez, ox, oy, oz);
}
