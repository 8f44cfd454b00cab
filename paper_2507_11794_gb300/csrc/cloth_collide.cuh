// Collision of a node's substep path with the surface model (device code
// shared by the stepping kernels and the adjoint's recompute).
//
// Broad phase (not in the paper, which tests every pair; a uniform grid over
// the surface triangles): the path S -> E is boxed and the triangles listed in
// the grid cells of that box are the candidates; a triangle listed in several
// of those cells is tested only in the first cell the two boxes share.
// Narrow phase: the extended Moller-Trumbore test of Section 3 on the path
// against each candidate.  Response (Algorithm 2): with K hits at
// distances t_k along r = (E - S)/|E - S|, the node moves to
// S + mean_k max(t_k - delta, 0) r and its velocity is scaled by the
// restitution factor.
#pragma once

#include "cloth_internal.h"

// Path of one node: start S, unit direction r, length L.
struct CollPath {
    float sx, sy, sz, rx, ry, rz, L;
};

// Grid-cell box of a path (cell_coord on both ends, per axis).
struct CollBox {
    int lox, loy, loz, hix, hiy, hiz;
};

__device__ __forceinline__ CollBox coll_box(const StepParams &p, float sx, float sy, float sz, float ex, float ey,
                                            float ez)
{
    CollBox b;
    b.lox = cell_coord(fminf(sx, ex), p.go[0], p.ginv, p.gd[0]);
    b.hix = cell_coord(fmaxf(sx, ex), p.go[0], p.ginv, p.gd[0]);
    b.loy = cell_coord(fminf(sy, ey), p.go[1], p.ginv, p.gd[1]);
    b.hiy = cell_coord(fmaxf(sy, ey), p.go[1], p.ginv, p.gd[1]);
    b.loz = cell_coord(fminf(sz, ez), p.go[2], p.ginv, p.gd[2]);
    b.hiz = cell_coord(fmaxf(sz, ez), p.go[2], p.ginv, p.gd[2]);
    return b;
}

// One candidate: grid entry e met in cell (cx, cy, cz) of a box whose low
// corner is (lox, loy, loz).  Returns true on a hit, with th the distance
// along r and f = 1/a (a = e1 . (r x e2)); A, B, C receive the triangle
// record (v0, e1, e2).
__device__ __forceinline__ bool coll_candidate(const StepParams &p, const CollPath &q, long long e, int cx, int cy,
                                               int cz, int lox, int loy, int loz, float &th, float &f, float4 &A,
                                               float4 &B, float4 &C)
{
    A = __ldg(p.etri + 3 * e);
    B = __ldg(p.etri + 3 * e + 1);
    C = __ldg(p.etri + 3 * e + 2);
    // the record's w lanes hold the low cell of the triangle's box
    if (max(__float_as_int(A.w), lox) != cx || max(__float_as_int(B.w), loy) != cy ||
        max(__float_as_int(C.w), loz) != cz)
        return false;
    // extended Moller-Trumbore: edge S -> E, direction r, length L
    const float hx = q.ry * C.z - q.rz * C.y;
    const float hy = q.rz * C.x - q.rx * C.z;
    const float hz = q.rx * C.y - q.ry * C.x;
    const float a = B.x * hx + B.y * hy + B.z * hz;
    if (fabsf(a) < p.eps) return false;
    f = 1.0f / a;
    const float qx0 = q.sx - A.x, qy0 = q.sy - A.y, qz0 = q.sz - A.z;
    const float u = f * (qx0 * hx + qy0 * hy + qz0 * hz);
    if (u < 0.0f || u > 1.0f) return false;
    const float qx = qy0 * B.z - qz0 * B.y;
    const float qy = qz0 * B.x - qx0 * B.z;
    const float qz = qx0 * B.y - qy0 * B.x;
    const float v = f * (q.rx * qx + q.ry * qy + q.rz * qz);
    th = f * (C.x * qx + C.y * qy + C.z * qz);
    if (v < 0.0f || u + v > 1.0f) return false;
    return th > p.tmin && th < q.L;
}

// Point S + th r of a path, each coordinate one rounded fused multiply-add,
// so every kernel that computes a hit point gets the same bits.
__device__ __forceinline__ float3 coll_hit_point(const CollPath &q, float th)
{
    return make_float3(__fmaf_rn(th, q.rx, q.sx), __fmaf_rn(th, q.ry, q.sy), __fmaf_rn(th, q.rz, q.sz));
}

// Path of S -> E; false when it is shorter than eps (no test).
__device__ __forceinline__ bool coll_path(const StepParams &p, float sx, float sy, float sz, float ex, float ey,
                                          float ez, CollPath &q)
{
    const float dx = ex - sx, dy = ey - sy, dz = ez - sz;
    q.L = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(q.L >= p.eps)) return false;
    q.sx = sx; q.sy = sy; q.sz = sz;
    q.rx = dx / q.L; q.ry = dy / q.L; q.rz = dz / q.L;
    return true;
}

// Broad + narrow phase and response of one node, one thread walking all
// candidates in (z, y, x) cell order and entry order.  On K > 0 hits returns
// true and the response position.  GRAD also returns, for the adjoint's
// recompute of an over-long path, mK = (m, K, r) with
// m = mean max(t_k - delta, 0), and over the active hits (t_k > delta) the
// sums g1 = sum n/a and g2 = sum t n/a (n = e1 x e2), the derivatives of t_k
// w.r.t. S and r.  The cooperative kernel below sums the same hits in the
// same order, so both see the same response.
template <bool GRAD>
__device__ __forceinline__ bool collide_t(const StepParams &p, float sx, float sy, float sz, float ex, float ey,
                                          float ez, float &ox, float &oy, float &oz, float *g1 = nullptr,
                                          float *g2 = nullptr, float *mK = nullptr)
{
    CollPath q;
    if (!coll_path(p, sx, sy, sz, ex, ey, ez, q)) return false;
    const CollBox bx = coll_box(p, sx, sy, sz, ex, ey, ez);
    int K = 0;
    float acc = 0.0f;
    for (int cz = bx.loz; cz <= bx.hiz; cz++)
        for (int cy = bx.loy; cy <= bx.hiy; cy++)
            for (int cx = bx.lox; cx <= bx.hix; cx++) {
                const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
                const int e0 = __ldg(p.cell_start + cell), e1 = __ldg(p.cell_start + cell + 1);
#pragma unroll 2
                for (int e = e0; e < e1; e++) {
                    float th, f;
                    float4 A, B, C;
                    if (!coll_candidate(p, q, e, cx, cy, cz, bx.lox, bx.loy, bx.loz, th, f, A, B, C)) continue;
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
        mK[2] = q.rx; mK[3] = q.ry; mK[4] = q.rz;
    }
    ox = sx + m * q.rx;
    oy = sy + m * q.ry;
    oz = sz + m * q.rz;
    return true;
}

// ------------------------------------------------- cooperative list pass
// The walk appends the nodes whose path box meets the box of the mesh's vertices.
// Most of them find empty cells; the few next to the surface find about a
// dozen candidates each, and those sit next to one another in the list.  One
// thread per node would leave those few threads testing their candidates one
// after another while the rest of the GPU idles, so each warp instead:
//  1. takes 32 list entries dealt round robin over all warps (entry i to warp
//     i mod #warps, spreading a run of neighbouring nodes over many warps),
//     boxes each path and counts its candidates over the box's cells;
//  2. spreads the warp's candidates over its 32 lanes, one test per lane and
//     round; each owner lane then adds its hits in candidate order (the
//     order collide_t uses, so the sum is the same float sum);
//  3. owner lanes apply the response.
// A path whose box spans more than COLL_MAXC cells (a node moving further
// than a cell in one substep) is handled by its own lane with collide_t.
constexpr int COLL_WARPS = 8;  // warps per CTA of the collision kernels
constexpr int COLL_MAXC = 8;   // cells of a box spread over the warp

struct CollLane {
    float4 s;                   // S, L
    float4 r;                   // r, owning cloth (int bits)
    int4 box;                   // low cell, x extent | y extent << 16
    int2 cell[COLL_MAXC];       // per cell of the box: first entry, end of the lane's running count
};

// Per-warp scratch of the cooperative pass, for a CTA of W warps.
template <int W>
struct CollSharedT {
    CollLane lane[W][32];
    int base[W][32];    // first candidate index of each lane (warp exclusive scan)
    float val[W][32];   // one round's results: max(t - delta, 0) on a hit, else -1
};
using CollShared = CollSharedT<COLL_WARPS>;
// The recording variant adds each candidate's terms of g1 and g2.
struct CollSharedRec : CollShared {
    float g[COLL_WARPS][6][32];
};

// Records the response data of a hit node at plane offset o for the reverse
// pass: m, r, g1 / K, g2 / K (the factors it multiplies by the adjoints) and
// the node's bit.
__device__ __forceinline__ void coll_record(const StepParams &p, long long o, float m, float K, float rx, float ry,
                                            float rz, const float g1[3], const float g2[3])
{
    const long long st = p.stride;
    const float invK = 1.0f / K;
    float *cd = p.cdata;
    cd[o] = m;
    cd[st + o] = rx;
    cd[2 * st + o] = ry;
    cd[3 * st + o] = rz;
    cd[4 * st + o] = g1[0] * invK;
    cd[5 * st + o] = g1[1] * invK;
    cd[6 * st + o] = g1[2] * invK;
    cd[7 * st + o] = g2[0] * invK;
    cd[8 * st + o] = g2[1] * invK;
    cd[9 * st + o] = g2[2] * invK;
    atomicOr(p.cbits + (o >> 5), 1u << (o & 31));
}

// Src supplies per list entry i: entry(i, cloth, offset) and params(cloth).
// REC (with CollSharedRec): also sums, over the active hits in the same
// order, g1 and g2 as collide_t<true> does and records them (coll_record).
// One round of the cooperative pass: every lane of the warp brings one entry
// (valid: whether it has one; i: its index for src.entry).  ntest (lane 0)
// accumulates the candidate triangles the warp tested, nhit (every lane) the
// nodes that hit.
// With has_pre the entry's offset is pre_o, loaded by the caller (cloth 0).
template <bool REC, class Src, class Sh>
__device__ __forceinline__ void collide_batch(const Src &src, Sh &sh, unsigned long long k, bool valid,
                                              unsigned long long i, float &fsum, unsigned &ntest, unsigned &nhit,
                                              bool has_pre = false, long long pre_o = 0)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    CollLane &me = sh.lane[wib][lane];
    {
        int cnt = 0, cloth = 0;
        bool serial = false;
        long long o = 0;
        float sx = 0.0f, sy = 0.0f, sz = 0.0f, ex = 0.0f, ey = 0.0f, ez = 0.0f;
        CollPath q;
        float *out = nullptr;
        long long st = 0;
        if (valid) {
            if (has_pre) o = pre_o;
            else src.entry(i, cloth, o);
            const StepParams &p = src.params(cloth);
            st = p.stride;
            const float *in = (k & 1ull) ? p.state1 : p.state0;
            out = (k & 1ull) ? p.state0 : p.state1;
            sx = __ldg(in + o); sy = __ldg(in + st + o); sz = __ldg(in + 2 * st + o);
            ex = out[o]; ey = out[st + o]; ez = out[2 * st + o];
            if (coll_path(p, sx, sy, sz, ex, ey, ez, q)) {
                const CollBox bx = coll_box(p, sx, sy, sz, ex, ey, ez);
                const int nxc = bx.hix - bx.lox + 1, nyc = bx.hiy - bx.loy + 1, nzc = bx.hiz - bx.loz + 1;
                if ((long long)nxc * nyc * nzc > COLL_MAXC) {
                    serial = true;
                } else {
                    int c = 0;
                    for (int cz = bx.loz; cz <= bx.hiz; cz++)
                        for (int cy = bx.loy; cy <= bx.hiy; cy++)
                            for (int cx = bx.lox; cx <= bx.hix; cx++, c++) {
                                const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
                                const int e0 = __ldg(p.cell_start + cell), e1 = __ldg(p.cell_start + cell + 1);
                                cnt += e1 - e0;
                                me.cell[c] = make_int2(e0, cnt);
                            }
                    me.s = make_float4(q.sx, q.sy, q.sz, q.L);
                    me.r = make_float4(q.rx, q.ry, q.rz, __int_as_float(cloth));
                    me.box = make_int4(bx.lox, bx.loy, bx.loz, nxc | (nyc << 16));
                }
            }
        }
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 0) ntest += (unsigned)total;
        const int excl = incl - cnt;
        sh.base[wib][lane] = excl;
        __syncwarp();
        float acc = 0.0f;
        int K = 0;
        float g1[3] = {0.0f, 0.0f, 0.0f}, g2[3] = {0.0f, 0.0f, 0.0f};
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int j = r0 + lane;
            float val = -1.0f;
            float gn[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (j < total) {
                // owner: the last lane whose first candidate is <= j (it has cnt > 0)
                int ow = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (sh.base[wib][ow + step] <= j) ow += step;
                const CollLane &L = sh.lane[wib][ow];
                const int loc = j - sh.base[wib][ow];
                int c = 0;
                while (L.cell[c].y <= loc) c++;
                const long long e = L.cell[c].x + (loc - (c ? L.cell[c - 1].y : 0));
                const int nxc = L.box.w & 0xffff, nyc = L.box.w >> 16;
                const int cx = L.box.x + c % nxc, cy = L.box.y + (c / nxc) % nyc, cz = L.box.z + c / (nxc * nyc);
                const CollPath lq = {L.s.x, L.s.y, L.s.z, L.r.x, L.r.y, L.r.z, L.s.w};
                const StepParams &lp = src.params(__float_as_int(L.r.w));
                float th, f;
                float4 A, B, C;
                if (coll_candidate(lp, lq, e, cx, cy, cz, L.box.x, L.box.y, L.box.z, th, f, A, B, C)) {
                    val = fmaxf(th - lp.delta, 0.0f);
                    if (REC) {
                        // the terms collide_t<true> adds for an active hit (t - delta > 0)
                        const float nx = B.y * C.z - B.z * C.y, ny = B.z * C.x - B.x * C.z,
                                    nz = B.x * C.y - B.y * C.x;
                        gn[0] = nx * f; gn[1] = ny * f; gn[2] = nz * f;
                        gn[3] = th * nx * f; gn[4] = th * ny * f; gn[5] = th * nz * f;
                    }
                }
            }
            sh.val[wib][lane] = val;
            if constexpr (REC) {
                if (val > 0.0f) {
#pragma unroll
                    for (int t = 0; t < 6; t++) sh.g[wib][t][lane] = gn[t];
                }
            }
            __syncwarp();
            if (cnt > 0) {
                const int q0 = max(excl, r0), q1 = min(excl + cnt, r0 + 32);
                for (int t = q0; t < q1; t++) {
                    const float v = sh.val[wib][t - r0];
                    if (v >= 0.0f) {
                        acc += v;
                        K++;
                        if constexpr (REC) {
                            if (v > 0.0f) {
                                g1[0] += sh.g[wib][0][t - r0]; g1[1] += sh.g[wib][1][t - r0];
                                g1[2] += sh.g[wib][2][t - r0];
                                g2[0] += sh.g[wib][3][t - r0]; g2[1] += sh.g[wib][4][t - r0];
                                g2[2] += sh.g[wib][5][t - r0];
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (!valid) return;
        const StepParams &p = src.params(cloth);
        float ox, oy, oz;
        bool hit;
        if (serial) {
            if (REC) {
                float sg1[3] = {0.0f, 0.0f, 0.0f}, sg2[3] = {0.0f, 0.0f, 0.0f}, mK[5];
                hit = collide_t<true>(p, sx, sy, sz, ex, ey, ez, ox, oy, oz, sg1, sg2, mK);
                if (hit) coll_record(p, o, mK[0], mK[1], mK[2], mK[3], mK[4], sg1, sg2);
            } else {
                hit = collide_t<false>(p, sx, sy, sz, ex, ey, ez, ox, oy, oz);
            }
        } else {
            hit = K > 0;
            if (hit) {
                const float m = acc / (float)K;
                ox = sx + m * q.rx;
                oy = sy + m * q.ry;
                oz = sz + m * q.rz;
                if (REC) coll_record(p, o, m, (float)K, q.rx, q.ry, q.rz, g1, g2);
            }
        }
        if (hit) {
            out[o] = ox;
            out[st + o] = oy;
            out[2 * st + o] = oz;
            out[3 * st + o] *= p.restitution;
            out[4 * st + o] *= p.restitution;
            out[5 * st + o] *= p.restitution;
            fsum += ox + oy + oz;
            nhit++;
        }
    }
}

// The cooperative pass over a list of n entries: entry i goes to warp
// i mod #warps (see above), 32 entries per warp and round.  has_pre: the
// lane's entry of the first round (index coll_first_index()) is pre_o, which
// the caller loaded before it knew n.
template <bool REC = false, class Src, class Sh>
__device__ __forceinline__ void collide_list(const Src &src, Sh &sh, unsigned long long k, unsigned n, float &fsum,
                                             unsigned &ntest, unsigned &nhit, bool has_pre = false,
                                             long long pre_o = 0)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long nw = (unsigned long long)gridDim.x * COLL_WARPS;
    const unsigned long long w = (unsigned long long)blockIdx.x * COLL_WARPS + wib;
    for (unsigned long long b0 = 0; b0 < n; b0 += 32ull * nw) {
        const unsigned long long i = b0 + (unsigned long long)lane * nw + w;
        collide_batch<REC>(src, sh, k, i < n, i, fsum, ntest, nhit, has_pre && b0 == 0, pre_o);
    }
}

// The calling lane's list index in the first round of collide_list.
__device__ __forceinline__ unsigned long long coll_first_index()
{
    const unsigned long long nw = (unsigned long long)gridDim.x * COLL_WARPS;
    return (unsigned long long)(threadIdx.x & 31) * nw + (unsigned long long)blockIdx.x * COLL_WARPS +
           (threadIdx.x >> 5);
}

// Adds a collision pass's counts to the cloth's running statistics: every
// warp's tested candidates and hit nodes are summed per CTA in shared memory
// (s2, zeroed by the caller before a __syncthreads), then one thread adds the
// CTA's totals; CTA 0 also adds the list length n.  The adds return nothing,
// so no thread waits on them.
__device__ __forceinline__ void coll_stats_add(DevCtrl *ctrl, unsigned *s2, unsigned n, unsigned ntest, unsigned nhit)
{
    const unsigned h = __reduce_add_sync(0xffffffffu, nhit);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s2[0], ntest);
        atomicAdd(&s2[1], h);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s2[0]) atomicAdd(&ctrl->stat_tested, (unsigned long long)s2[0]);
        if (s2[1]) atomicAdd(&ctrl->stat_hits, (unsigned long long)s2[1]);
        if (blockIdx.x == 0) atomicAdd(&ctrl->stat_listed, (unsigned long long)n);
    }
}

// ------------------------------------------- edge-triangle narrow phase
// The paper's own narrow phase (Section 3): edges of the cloth triangles (the
// grid's quads split along their (r,c)-(r+1,c+1) diagonal) at the updated
// positions against the surface triangles.  A hit of an edge at P affects
// every vertex of the cloth triangles that share the edge; an affected free
// node i gets the direction from its previous position S_i towards P,
// stopping delta short, max(|P - S_i| - delta, 0) (P - S_i)/|P - S_i|, and
// moves by the mean over its hits (Algorithm 2).  Gathered per node: the 12
// edges whose triangles contain node (r, c), each as (owner endpoint ->
// other endpoint) with the owner the edge's upper-left node, the orientation
// the test's arithmetic is defined in.
struct EdgeOfs {
    signed char ar, ac, br, bc;
};
__device__ __forceinline__ EdgeOfs edge_of_node(int q)
{
    // (0,+1) edges: own, left, up-left row above, row below
    // (+1,0) edges: own, above, up-left column, right column
    // (+1,+1) edges: own, up-left, the two that have (r,c) as opposite vertex
    switch (q) {
    case 0: return {0, 0, 0, 1};
    case 1: return {0, -1, 0, 0};
    case 2: return {-1, -1, -1, 0};
    case 3: return {1, 0, 1, 1};
    case 4: return {0, 0, 1, 0};
    case 5: return {-1, 0, 0, 0};
    case 6: return {-1, -1, 0, -1};
    case 7: return {0, 1, 1, 1};
    case 8: return {0, 0, 1, 1};
    case 9: return {-1, -1, 0, 0};
    case 10: return {-1, 0, 0, 1};
    default: return {0, -1, 1, 0};
    }
}
constexpr int EDGES_PER_NODE = 12;
// Hits after an edge's first whose points pass A stores (p.edge_more); pass B
// walks an edge with more hits than 1 + EDGE_MORE again.
constexpr int EDGE_MORE = CLOTH_EDGE_MORE;

struct EdgeShared {
    CollLane lane[COLL_WARPS][32];
    int base[COLL_WARPS][32];
    float4 hit[COLL_WARPS][32];  // one round's results: hit point P and 1, or w = 0
};

// The kind of the triangulation edge from (ra, ca) to (rb, cb): 0 (0,+1),
// 1 (+1,0), 2 (+1,+1).
__device__ __forceinline__ int edge_kind(int ra, int ca, int rb, int cb) { return rb == ra ? 0 : (cb == ca ? 1 : 2); }

// The first hit point of an edge path and its number of hits, walked by the
// whole warp (every lane passes the same path and box; call from converged
// code): the box's cells 32 at a time, x fastest, and each chunk's candidates
// 32 at a time in cell order, so the first hit and the count are those of a
// walk over the candidates in order.  Returns the same record on every lane
// and adds the candidates tested to ntest.
__device__ __forceinline__ float4 edge_hits_warp(const StepParams &p, const CollPath &path, const CollBox &bx,
                                                 long long slot, int lane, unsigned &ntest)
{
    constexpr unsigned FULLW = 0xffffffffu;
    const int nxc = bx.hix - bx.lox + 1, nyc = bx.hiy - bx.loy + 1, nzc = bx.hiz - bx.loz + 1;
    const long long nxy = (long long)nxc * nyc, ncell = nxy * nzc;
    float4 rec = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (long long c0 = 0; c0 < ncell; c0 += 32) {
        const long long cc = c0 + lane;
        int e0 = 0, cnt = 0, cx = 0, cy = 0, cz = 0;
        if (cc < ncell) {
            cz = bx.loz + (int)(cc / nxy);
            const int rem = (int)(cc - (long long)(cz - bx.loz) * nxy);
            cy = bx.loy + rem / nxc;
            cx = bx.lox + rem % nxc;
            const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
            e0 = __ldg(p.cell_start + cell);
            cnt = __ldg(p.cell_start + cell + 1) - e0;
        }
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(FULLW, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(FULLW, incl, 31);
        const int excl = incl - cnt;
        ntest += (unsigned)total;
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int j = r0 + lane;
            // the lane whose cell holds candidate j: the last with excl <= j
            int ow = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(FULLW, excl, ow + step) <= j) ow += step;
            const int oe0 = __shfl_sync(FULLW, e0, ow), oex = __shfl_sync(FULLW, excl, ow);
            const int ocx = __shfl_sync(FULLW, cx, ow), ocy = __shfl_sync(FULLW, cy, ow),
                      ocz = __shfl_sync(FULLW, cz, ow);
            bool hit = false;
            float th = 0.0f;
            if (j < total) {
                float f;
                float4 A, B, C;
                hit = coll_candidate(p, path, (long long)oe0 + (j - oex), ocx, ocy, ocz, bx.lox, bx.loy, bx.loz, th,
                                     f, A, B, C);
            }
            const unsigned hm = __ballot_sync(FULLW, hit);
            if (hm) {
                const float3 hp = coll_hit_point(path, th);
                const float hx = hp.x, hy = hp.y, hz = hp.z;
                // this lane's hit is number rank (from 0) of the edge
                const int rank = (int)rec.w + __popc(hm & ((1u << lane) - 1u));
                if (hit && rank >= 1 && rank <= EDGE_MORE)
                    p.edge_more[(long long)(rank - 1) * 3 * p.stride + slot] = make_float4(hx, hy, hz, 1.0f);
                if (rec.w == 0.0f) {
                    const int src = __ffs(hm) - 1;
                    rec = make_float4(__shfl_sync(FULLW, hx, src), __shfl_sync(FULLW, hy, src),
                                      __shfl_sync(FULLW, hz, src), 0.0f);
                }
                rec.w += (float)__popc(hm);
            }
        }
    }
    return rec;
}

// Pass A of the edge narrow phase: every listed node tests the three edges it
// owns, (0,+1), (+1,0) and (+1,+1) from it (the triangulation's edges,
// oriented from their upper-left endpoint), at the updated positions, so each
// edge is tested once.  32 edges per warp and round, their candidates spread
// over the lanes as in the node pass; an edge whose box spans more than
// COLL_MAXC cells is walked afterwards by the whole warp (edge_hits_warp).
// Records per edge its first hit point (in candidate order) and its number of
// hits, p.edge_hit[kind * stride + owner] = (P, K), and the points of its hits
// 2 .. 1 + EDGE_MORE at p.edge_more[(h - 2) * 3 * stride + kind * stride +
// owner].  Counts the lane's tested candidates and edges that hit into ntest
// and nhit.
__device__ __forceinline__ void edge_test_list(const StepParams &p, EdgeShared &sh, unsigned long long k, unsigned n,
                                               unsigned &ntest, unsigned &nhit)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long nw = (unsigned long long)gridDim.x * COLL_WARPS;
    const unsigned long long w = (unsigned long long)blockIdx.x * COLL_WARPS + wib;
    CollLane &me = sh.lane[wib][lane];
    const long long st = p.stride;
    const float *xs = (k & 1ull) ? p.state0 : p.state1;  // updated positions (written by the walk)
    const unsigned long long items = 3ull * n;
    for (unsigned long long b0 = 0; b0 < items; b0 += 32ull * nw) {
        const unsigned long long j = b0 + (unsigned long long)lane * nw + w;
        int cnt = 0;
        bool has = false, wide = false;
        long long slot = 0;
        float4 rec = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        CollPath path = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        CollBox bx = {0, 0, 0, 0, 0, 0};
        if (j < items) {
            const int q = (int)(j % 3ull);
            const int o = __ldg(p.coll_list + j / 3ull);
            const int r = o / p.pitch, c = o - r * p.pitch;
            const int rb = r + (q >= 1 ? 1 : 0), cb = c + (q != 1 ? 1 : 0);
            if (rb < p.ny && cb < p.nx) {
                has = true;
                slot = (long long)q * st + o;
                const long long ob = (long long)rb * p.pitch + cb;
                const float x0 = xs[o], y0 = xs[st + o], z0 = xs[2 * st + o];
                const float x1 = xs[ob], y1 = xs[st + ob], z1 = xs[2 * st + ob];
                if (coll_path(p, x0, y0, z0, x1, y1, z1, path)) {
                    bx = coll_box(p, x0, y0, z0, x1, y1, z1);
                    const int nxc = bx.hix - bx.lox + 1, nyc = bx.hiy - bx.loy + 1, nzc = bx.hiz - bx.loz + 1;
                    if ((long long)nxc * nyc * nzc <= COLL_MAXC) {
                        int cc = 0;
                        for (int cz = bx.loz; cz <= bx.hiz; cz++)
                            for (int cy = bx.loy; cy <= bx.hiy; cy++)
                                for (int cx = bx.lox; cx <= bx.hix; cx++, cc++) {
                                    const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
                                    const int e0 = __ldg(p.cell_start + cell), e1 = __ldg(p.cell_start + cell + 1);
                                    cnt += e1 - e0;
                                    me.cell[cc] = make_int2(e0, cnt);
                                }
                        me.s = make_float4(path.sx, path.sy, path.sz, path.L);
                        me.r = make_float4(path.rx, path.ry, path.rz, 0.0f);
                        me.box = make_int4(bx.lox, bx.loy, bx.loz, nxc | (nyc << 16));
                    } else {
                        wide = true;
                    }
                }
            }
        }
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - cnt;
        sh.base[wib][lane] = excl;
        __syncwarp();
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int jj = r0 + lane;
            float4 hv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (jj < total) {
                int ow = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (sh.base[wib][ow + step] <= jj) ow += step;
                const CollLane &L = sh.lane[wib][ow];
                const int loc = jj - sh.base[wib][ow];
                int cc = 0;
                while (L.cell[cc].y <= loc) cc++;
                const long long e = L.cell[cc].x + (loc - (cc ? L.cell[cc - 1].y : 0));
                const int nxc = L.box.w & 0xffff, nyc = L.box.w >> 16;
                const int cx = L.box.x + cc % nxc, cy = L.box.y + (cc / nxc) % nyc, cz = L.box.z + cc / (nxc * nyc);
                const CollPath lq = {L.s.x, L.s.y, L.s.z, L.r.x, L.r.y, L.r.z, L.s.w};
                float th, f;
                float4 A, B, C;
                if (coll_candidate(p, lq, e, cx, cy, cz, L.box.x, L.box.y, L.box.z, th, f, A, B, C)) {
                    const float3 hp = coll_hit_point(lq, th);
                    hv = make_float4(hp.x, hp.y, hp.z, 1.0f);
                }
            }
            sh.hit[wib][lane] = hv;
            __syncwarp();
            if (cnt > 0) {
                const int q0 = max(excl, r0), q1 = min(excl + cnt, r0 + 32);
                for (int t = q0; t < q1; t++) {
                    const float4 P = sh.hit[wib][t - r0];
                    if (P.w == 0.0f) continue;
                    if (rec.w == 0.0f) rec = make_float4(P.x, P.y, P.z, 0.0f);
                    else if (rec.w <= (float)EDGE_MORE) p.edge_more[(long long)(rec.w - 1.0f) * 3 * st + slot] = P;
                    rec.w += 1.0f;
                }
            }
            __syncwarp();
        }
        // the wide edges of this round, one at a time over the whole warp
        for (unsigned wm = __ballot_sync(0xffffffffu, wide); wm; wm &= wm - 1u) {
            const int src = __ffs(wm) - 1;
            const CollPath q = {__shfl_sync(0xffffffffu, path.sx, src), __shfl_sync(0xffffffffu, path.sy, src),
                                __shfl_sync(0xffffffffu, path.sz, src), __shfl_sync(0xffffffffu, path.rx, src),
                                __shfl_sync(0xffffffffu, path.ry, src), __shfl_sync(0xffffffffu, path.rz, src),
                                __shfl_sync(0xffffffffu, path.L, src)};
            const CollBox b = {__shfl_sync(0xffffffffu, bx.lox, src), __shfl_sync(0xffffffffu, bx.loy, src),
                               __shfl_sync(0xffffffffu, bx.loz, src), __shfl_sync(0xffffffffu, bx.hix, src),
                               __shfl_sync(0xffffffffu, bx.hiy, src), __shfl_sync(0xffffffffu, bx.hiz, src)};
            const long long sl = __shfl_sync(0xffffffffu, slot, src);
            unsigned t = 0;
            const float4 wr = edge_hits_warp(p, q, b, sl, lane, t);
            if (lane == src) {
                rec = wr;
                ntest += t;
            }
        }
        ntest += (unsigned)cnt;
        nhit += rec.w > 0.0f ? 1u : 0u;
        if (has) p.edge_hit[slot] = rec;
    }
}

// Running sum of one node's response directions (Algorithm 2): adds the
// direction from S towards the hit point P, stopping delta short.
struct EdgeAcc {
    float ax, ay, az;
    int K;
};
__device__ __forceinline__ void edge_acc_add(EdgeAcc &a, float delta, float sx, float sy, float sz, float Px,
                                             float Py, float Pz)
{
    const float wx = Px - sx, wy = Py - sy, wz = Pz - sz;
    const float lw = sqrtf(wx * wx + wy * wy + wz * wz);
    const float sc = lw > 0.0f ? fmaxf(lw - delta, 0.0f) / lw : 0.0f;
    a.ax += sc * wx;
    a.ay += sc * wy;
    a.az += sc * wz;
    a.K++;
}

// An edge with more hits than pass A stored: walks its candidates again, in
// order, and adds every hit after the first (already added).  Out of line:
// rare, and it keeps the gather's unrolled loop small.
static __device__ __noinline__ EdgeAcc edge_rewalk(const StepParams &p, const float *xs, long long oa, long long ob,
                                                   float sx, float sy, float sz, EdgeAcc a)
{
    const long long st = p.stride;
    const float x0 = xs[oa], y0 = xs[st + oa], z0 = xs[2 * st + oa];
    const float x1 = xs[ob], y1 = xs[st + ob], z1 = xs[2 * st + ob];
    CollPath path;
    if (!coll_path(p, x0, y0, z0, x1, y1, z1, path)) return a;
    const CollBox bx = coll_box(p, x0, y0, z0, x1, y1, z1);
    bool first = true;
    for (int cz = bx.loz; cz <= bx.hiz; cz++)
        for (int cy = bx.loy; cy <= bx.hiy; cy++)
            for (int cx = bx.lox; cx <= bx.hix; cx++) {
                const long long cell = ((long long)cz * p.gd[1] + cy) * p.gd[0] + cx;
                const int e0 = __ldg(p.cell_start + cell), e1 = __ldg(p.cell_start + cell + 1);
                for (int ee = e0; ee < e1; ee++) {
                    float th, f;
                    float4 A, B, C;
                    if (!coll_candidate(p, path, ee, cx, cy, cz, bx.lox, bx.loy, bx.loz, th, f, A, B, C)) continue;
                    if (first) {
                        first = false;
                        continue;
                    }
                    const float3 hp = coll_hit_point(path, th);
                    edge_acc_add(a, p.delta, sx, sy, sz, hp.x, hp.y, hp.z);
                }
            }
    return a;
}

// Pass B: every listed free node gathers the hits of the 12 edges whose
// triangles contain it (in the order of edge_of_node, each edge's hits in
// candidate order) and writes its response to p.edge_resp[i]: (position, 1),
// or zeros without a hit.  An edge whose owner was not listed this substep
// (stamp) cannot hit.  The stamps, then the records, of the 12 edges are
// loaded before any is used; an edge with more than 1 + EDGE_MORE hits is
// walked again (edge_rewalk).
__device__ __forceinline__ void edge_gather_list(const StepParams &p, unsigned long long k, unsigned n)
{
    const long long st = p.stride;
    const float *in = (k & 1ull) ? p.state1 : p.state0;
    const float *xs = (k & 1ull) ? p.state0 : p.state1;
    const unsigned long long stamp = k + 1ull;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = __ldg(p.coll_list + i);
        const bool pinned = p.pin_bits && ((__ldg(p.pin_bits + (o >> 5)) >> (o & 31)) & 1u);
        float4 resp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (!pinned) {
            const int r = o / p.pitch, c = o - r * p.pitch;
            const float sx = __ldg(in + o), sy = __ldg(in + st + o), sz = __ldg(in + 2 * st + o);
            bool live[EDGES_PER_NODE];
#pragma unroll
            for (int q = 0; q < EDGES_PER_NODE; q++) {
                const EdgeOfs e = edge_of_node(q);
                const int ra = r + e.ar, ca = c + e.ac, rb = r + e.br, cb = c + e.bc;
                const bool inside = ra >= 0 && ca >= 0 && rb < p.ny && cb < p.nx && ca < p.nx && cb >= 0;
                live[q] = inside && p.edge_stamp[inside ? (long long)ra * p.pitch + ca : 0] == stamp;
            }
            float4 rec[EDGES_PER_NODE];
#pragma unroll
            for (int q = 0; q < EDGES_PER_NODE; q++) {
                const EdgeOfs e = edge_of_node(q);
                const long long slot = (long long)edge_kind(e.ar, e.ac, e.br, e.bc) * st +
                                       (long long)(r + e.ar) * p.pitch + (c + e.ac);
                rec[q] = live[q] ? p.edge_hit[slot] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            EdgeAcc acc = {0.0f, 0.0f, 0.0f, 0};
#pragma unroll
            for (int q = 0; q < EDGES_PER_NODE; q++) {
                const float4 rq = rec[q];
                if (rq.w == 0.0f) continue;
                edge_acc_add(acc, p.delta, sx, sy, sz, rq.x, rq.y, rq.z);
                if (rq.w == 1.0f) continue;
                const EdgeOfs e = edge_of_node(q);
                const long long oa = (long long)(r + e.ar) * p.pitch + (c + e.ac);
                if (rq.w <= (float)(1 + EDGE_MORE)) {
                    const long long slot = (long long)edge_kind(e.ar, e.ac, e.br, e.bc) * st + oa;
                    for (int h = 1; h < (int)rq.w; h++) {
                        const float4 P = p.edge_more[(long long)(h - 1) * 3 * st + slot];
                        edge_acc_add(acc, p.delta, sx, sy, sz, P.x, P.y, P.z);
                    }
                } else {
                    const long long ob = (long long)(r + e.br) * p.pitch + (c + e.bc);
                    acc = edge_rewalk(p, xs, oa, ob, sx, sy, sz, acc);
                }
            }
            if (acc.K > 0)
                resp = make_float4(sx + acc.ax / (float)acc.K, sy + acc.ay / (float)acc.K, sz + acc.az / (float)acc.K,
                                   1.0f);
        }
        p.edge_resp[i] = resp;
    }
}
