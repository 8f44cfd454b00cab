// Uniform grid over the static surface triangles (the broad phase the paper
// lists as future work: it tests all triangle pairs, Section 3; culling and
// BVH are named in Section 5).  Built once per mesh as a counting sort of
// (cell, triangle) pairs:
//   1. per triangle: float32 AABB -> cell box (the float32 cell formula),
//      MT record (v0, e1 = v1 - v0, e2 = v2 - v0) and its pair count;
//   2. per-cell counts (atomics; counts are order independent);
//   3. exclusive prefix scan of the counts (warp-shuffle scans inside a
//      three-phase reduce / scan-of-sums / scan kernel) -> cell_start;
//   4. scatter of the triangle ids, then each cell's short list is sorted so
//      that the lists are ascending and the result is deterministic.
#include <math.h>
#include <stdio.h>

#include "cloth_internal.h"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void tri_prep_kernel(const float *__restrict__ verts, const int *__restrict__ tris, int nt, float ox,
                                float oy, float oz, float inv, int dx, int dy, int dz, float4 *__restrict__ rec,
                                int4 *__restrict__ box_hi, unsigned long long *__restrict__ total)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (t < nt) {
        const int i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
        const float ax = verts[3 * i0], ay = verts[3 * i0 + 1], az = verts[3 * i0 + 2];
        const float bx = verts[3 * i1], by = verts[3 * i1 + 1], bz = verts[3 * i1 + 2];
        const float cx = verts[3 * i2], cy = verts[3 * i2 + 1], cz = verts[3 * i2 + 2];
        const int lx = cell_coord(fminf(fminf(ax, bx), cx), ox, inv, dx);
        const int ly = cell_coord(fminf(fminf(ay, by), cy), oy, inv, dy);
        const int lz = cell_coord(fminf(fminf(az, bz), cz), oz, inv, dz);
        const int hx = cell_coord(fmaxf(fmaxf(ax, bx), cx), ox, inv, dx);
        const int hy = cell_coord(fmaxf(fmaxf(ay, by), cy), oy, inv, dy);
        const int hz = cell_coord(fmaxf(fmaxf(az, bz), cz), oz, inv, dz);
        rec[3 * t] = make_float4(ax, ay, az, __int_as_float(lx));
        rec[3 * t + 1] = make_float4(__fsub_rn(bx, ax), __fsub_rn(by, ay), __fsub_rn(bz, az), __int_as_float(ly));
        rec[3 * t + 2] = make_float4(__fsub_rn(cx, ax), __fsub_rn(cy, ay), __fsub_rn(cz, az), __int_as_float(lz));
        box_hi[t] = make_int4(hx, hy, hz, 0);
        cnt = (unsigned long long)(hx - lx + 1) * (unsigned long long)(hy - ly + 1) * (unsigned long long)(hz - lz + 1);
    }
    // warp-reduce the pair counts before one atomic per warp
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(total, cnt);
}

__global__ void cell_count_kernel(const float4 *__restrict__ rec, const int4 *__restrict__ box_hi, int nt, int dx,
                                  int dy, unsigned *__restrict__ cnt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int lx = __float_as_int(rec[3 * t].w), ly = __float_as_int(rec[3 * t + 1].w),
              lz = __float_as_int(rec[3 * t + 2].w);
    const int4 hi = box_hi[t];
    for (int z = lz; z <= hi.z; z++)
        for (int y = ly; y <= hi.y; y++)
            for (int x = lx; x <= hi.x; x++) atomicAdd(cnt + ((long long)z * dy + y) * dx + x, 1u);
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive scan of one CTA tile held as SCAN_ITEMS consecutive items per
// thread; returns the thread's exclusive prefix, *tile_sum the tile total.
__device__ unsigned block_excl_scan(unsigned thread_sum, unsigned *tile_sum)
{
    __shared__ unsigned warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned inc = warp_incl_scan(thread_sum);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0u;
        unsigned ti = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;
        if (lane == SCAN_THREADS / 32 - 1) *tile_sum = ti;
    }
    __syncthreads();
    const unsigned r = warp_tot[w] + inc - thread_sum;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const unsigned *__restrict__ in, long long n,
                                                                   unsigned *__restrict__ tile_sums)
{
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++)
        if (base + j < n) s += in[base + j];
    __shared__ unsigned tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the tile sums in place (any count).
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_kernel(unsigned *__restrict__ sums, long long nt)
{
    __shared__ unsigned tot;
    unsigned carry = 0;
    for (long long b = 0; b < nt; b += SCAN_TILE) {
        const long long base = b + threadIdx.x * SCAN_ITEMS;
        unsigned v[SCAN_ITEMS], s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            v[j] = base + j < nt ? sums[base + j] : 0u;
            s += v[j];
        }
        unsigned ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            if (base + j < nt) sums[base + j] = ex;
            ex += v[j];
        }
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_final_kernel(const unsigned *__restrict__ in, long long n,
                                                                  const unsigned *__restrict__ tile_off,
                                                                  int *__restrict__ out)
{
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        v[j] = base + j < n ? in[base + j] : 0u;
        s += v[j];
    }
    __shared__ unsigned tot;
    unsigned ex = block_excl_scan(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < n) out[base + j] = (int)ex;
        ex += v[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = (int)ex;
}

__global__ void cell_fill_kernel(const float4 *__restrict__ rec, const int4 *__restrict__ box_hi, int nt, int dx,
                                 int dy, const int *__restrict__ cell_start, unsigned *__restrict__ cursor,
                                 int *__restrict__ tri_ids)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int lx = __float_as_int(rec[3 * t].w), ly = __float_as_int(rec[3 * t + 1].w),
              lz = __float_as_int(rec[3 * t + 2].w);
    const int4 hi = box_hi[t];
    for (int z = lz; z <= hi.z; z++)
        for (int y = ly; y <= hi.y; y++)
            for (int x = lx; x <= hi.x; x++) {
                const long long c = ((long long)z * dy + y) * dx + x;
                const unsigned slot = atomicAdd(cursor + c, 1u);
                tri_ids[cell_start[c] + slot] = t;
            }
}

// Sort each cell's (short) list ascending: insertion sort by one thread.
__global__ void cell_sort_kernel(const int *__restrict__ cell_start, long long ncells, int *__restrict__ tri_ids)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int b = cell_start[c], e = cell_start[c + 1];
    for (int i = b + 1; i < e; i++) {
        const int key = tri_ids[i];
        int j = i - 1;
        while (j >= b && tri_ids[j] > key) {
            tri_ids[j + 1] = tri_ids[j];
            j--;
        }
        tri_ids[j + 1] = key;
    }
}

// Expand the sorted (cell, triangle) pairs into per-entry records read by the
// narrow phase without an indirection: the triangle's plane and first cell.
__global__ void expand_kernel(const float4 *__restrict__ rec, const int *__restrict__ tri_ids, long long n,
                              float4 *__restrict__ etri)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int t = tri_ids[e];
    etri[3 * e] = rec[3 * t];
    etri[3 * e + 1] = rec[3 * t + 1];
    etri[3 * e + 2] = rec[3 * t + 2];
}

__global__ void query_kernel(const float4 *__restrict__ rec, const int *__restrict__ cell_start,
                             const int *__restrict__ tri_ids, float ox, float oy, float oz, float inv, int dx, int dy,
                             int dz, const float *__restrict__ S, const float *__restrict__ E, int nseg,
                             int *__restrict__ counts, int *__restrict__ ids, int cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    const float sx = S[3 * i], sy = S[3 * i + 1], sz = S[3 * i + 2];
    const float ex = E[3 * i], ey = E[3 * i + 1], ez = E[3 * i + 2];
    const int lx = cell_coord(fminf(sx, ex), ox, inv, dx), hx = cell_coord(fmaxf(sx, ex), ox, inv, dx);
    const int ly = cell_coord(fminf(sy, ey), oy, inv, dy), hy = cell_coord(fmaxf(sy, ey), oy, inv, dy);
    const int lz = cell_coord(fminf(sz, ez), oz, inv, dz), hz = cell_coord(fmaxf(sz, ez), oz, inv, dz);
    int n = 0;
    for (int z = lz; z <= hz; z++)
        for (int y = ly; y <= hy; y++)
            for (int x = lx; x <= hx; x++) {
                const long long c = ((long long)z * dy + y) * dx + x;
                for (int e = cell_start[c]; e < cell_start[c + 1]; e++) {
                    const int t = tri_ids[e];
                    if (max(__float_as_int(rec[3 * t].w), lx) != x || max(__float_as_int(rec[3 * t + 1].w), ly) != y ||
                        max(__float_as_int(rec[3 * t + 2].w), lz) != z)
                        continue;
                    if (n < cap) ids[(long long)i * cap + n] = t;
                    n++;
                }
            }
    counts[i] = n;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int grid_params(const float *verts, const int32_t *tris, int32_t nt, float *h_out, float origin[3], int dims[3],
                float *inv_out)
{
    // h = (float)(2 * mean longest AABB side), summed in double in triangle
    // order; origin = (float)(min - 1.5h); dims = floor(extent/h) + 4; the cell
    // size doubles while the grid would exceed 2^24 cells.
    if (nt <= 0) return -1;
    double sum = 0.0;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t t = 0; t < nt; t++) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int j = 0; j < 3; j++) {
            const float *q = verts + 3 * (long long)tris[3 * (long long)t + j];
            for (int a = 0; a < 3; a++) {
                lo[a] = q[a] < lo[a] ? q[a] : lo[a];
                hi[a] = q[a] > hi[a] ? q[a] : hi[a];
            }
        }
        double side = 0.0;
        for (int a = 0; a < 3; a++) {
            const double e = (double)hi[a] - (double)lo[a];
            side = e > side ? e : side;
            mn[a] = lo[a] < mn[a] ? lo[a] : mn[a];
            mx[a] = hi[a] > mx[a] ? hi[a] : mx[a];
        }
        sum += side;
    }
    float h = (float)(2.0 * (sum / (double)nt));
    if (!(h > 0.0f)) h = 1.0f;
    for (;;) {
        long long cells = 1;
        for (int a = 0; a < 3; a++) {
            origin[a] = (float)((double)mn[a] - 1.5 * (double)h);
            dims[a] = (int)floor(((double)mx[a] - (double)mn[a]) / (double)h) + 4;
            cells *= dims[a];
        }
        if (cells <= (1ll << 24)) break;
        h = h * 2.0f;
    }
    *h_out = h;
    *inv_out = (float)(1.0 / (double)h);
    return 0;
}

#define GTRY(x)                          \
    do {                                 \
        cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) {         \
            err = e_;                    \
            goto done;                   \
        }                                \
    } while (0)

cudaError_t grid_build(const float *d_verts, const int *d_tris, int nt, DevGrid *g, cudaStream_t s)
{
    cudaError_t err = cudaSuccess;
    int4 *box_hi = nullptr;
    unsigned *cnt = nullptr, *cursor = nullptr, *sums = nullptr;
    unsigned long long *total = nullptr;
    unsigned long long htotal = 0;
    const long long nc = (long long)g->dims[0] * g->dims[1] * g->dims[2];
    const long long ntiles = (nc + SCAN_TILE - 1) / SCAN_TILE;
    g->ncells = nc;
    g->ntris = nt;
    g->tri = nullptr;
    g->cell_start = nullptr;
    g->tri_ids = nullptr;
    g->etri = nullptr;
    GTRY(cudaMalloc(&g->tri, sizeof(float4) * 3 * (size_t)nt));
    GTRY(cudaMalloc(&g->cell_start, sizeof(int) * (size_t)(nc + 1)));
    GTRY(cudaMalloc(&box_hi, sizeof(int4) * (size_t)nt));
    GTRY(cudaMalloc(&cnt, sizeof(unsigned) * (size_t)nc));
    GTRY(cudaMalloc(&cursor, sizeof(unsigned) * (size_t)nc));
    GTRY(cudaMalloc(&sums, sizeof(unsigned) * (size_t)ntiles));
    GTRY(cudaMalloc(&total, sizeof(unsigned long long)));
    GTRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (size_t)nc, s));
    GTRY(cudaMemsetAsync(cursor, 0, sizeof(unsigned) * (size_t)nc, s));
    GTRY(cudaMemsetAsync(total, 0, sizeof(unsigned long long), s));
    tri_prep_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(d_verts, d_tris, nt, g->origin[0], g->origin[1], g->origin[2],
                                                        g->inv, g->dims[0], g->dims[1], g->dims[2], g->tri, box_hi,
                                                        total);
    GTRY(cudaGetLastError());
    GTRY(cudaMemcpyAsync(&htotal, total, sizeof(htotal), cudaMemcpyDeviceToHost, s));
    GTRY(cudaStreamSynchronize(s));
    if (htotal >= 0x7fffffffull) {
        err = cudaErrorInvalidValue;  // reported as CLOTH_ERR_BAD_MESH by the caller
        goto done;
    }
    g->nentries = (long long)htotal;
    GTRY(cudaMalloc(&g->tri_ids, sizeof(int) * (size_t)(htotal > 0 ? htotal : 1)));
    cell_count_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(g->tri, box_hi, nt, g->dims[0], g->dims[1], cnt);
    GTRY(cudaGetLastError());
    scan_reduce_kernel<<<(int)ntiles, SCAN_THREADS, 0, s>>>(cnt, nc, sums);
    GTRY(cudaGetLastError());
    scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(sums, ntiles);
    GTRY(cudaGetLastError());
    scan_final_kernel<<<(int)ntiles, SCAN_THREADS, 0, s>>>(cnt, nc, sums, g->cell_start);
    GTRY(cudaGetLastError());
    cell_fill_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(g->tri, box_hi, nt, g->dims[0], g->dims[1], g->cell_start,
                                                         cursor, g->tri_ids);
    GTRY(cudaGetLastError());
    cell_sort_kernel<<<blocks_for(nc, 256), 256, 0, s>>>(g->cell_start, nc, g->tri_ids);
    GTRY(cudaGetLastError());
    GTRY(cudaMalloc(&g->etri, sizeof(float4) * 3 * (size_t)(htotal > 0 ? htotal : 1)));
    if (htotal > 0) {
        expand_kernel<<<blocks_for((long long)htotal, 256), 256, 0, s>>>(g->tri, g->tri_ids, (long long)htotal, g->etri);
        GTRY(cudaGetLastError());
    }
    GTRY(cudaStreamSynchronize(s));
done:
    cudaFree(box_hi);
    cudaFree(cnt);
    cudaFree(cursor);
    cudaFree(sums);
    cudaFree(total);
    if (err != cudaSuccess) grid_free(g);
    return err;
}

void grid_free(DevGrid *g)
{
    cudaFree(g->tri);
    cudaFree(g->cell_start);
    cudaFree(g->tri_ids);
    cudaFree(g->etri);
    g->etri = nullptr;
    g->tri = nullptr;
    g->cell_start = nullptr;
    g->tri_ids = nullptr;
    g->ntris = 0;
    g->nentries = 0;
}

cudaError_t grid_query(const DevGrid &g, const float *dS, const float *dE, int nseg, int *counts, int *ids, int cap,
                       cudaStream_t s)
{
    query_kernel<<<blocks_for(nseg, 128), 128, 0, s>>>(g.tri, g.cell_start, g.tri_ids, g.origin[0], g.origin[1],
                                                       g.origin[2], g.inv, g.dims[0], g.dims[1], g.dims[2], dS, dE,
                                                       nseg, counts, ids, cap);
    return cudaGetLastError();
}

// Grid build with every temporary buffer supplied by the caller (no
// allocation).  Same kernels and order as grid_build.  Writes the pair count
// to *nentries after the counting pass; when it exceeds entry_cap, or int32
// offsets (2^31 - 1 or more), nothing more is written and *done is false.
// Synchronises s.
cudaError_t grid_build_noalloc(const float *d_verts, const int *d_tris, int nt, const float origin[3], float inv,
                               const int dims[3], float4 *rec, int *cell_start, int *tri_ids, long long entry_cap,
                               int4 *box_hi, unsigned *cnt, unsigned *cursor, unsigned *sums,
                               unsigned long long *total, long long *nentries, bool *done, cudaStream_t s)
{
    const long long nc = (long long)dims[0] * dims[1] * dims[2];
    const long long ntiles = (nc + SCAN_TILE - 1) / SCAN_TILE;
    unsigned long long htotal = 0;
    cudaError_t e;
    *done = false;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (size_t)nc, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * (size_t)nc, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    tri_prep_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(d_verts, d_tris, nt, origin[0], origin[1], origin[2], inv,
                                                        dims[0], dims[1], dims[2], rec, box_hi, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&htotal, total, sizeof(htotal), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *nentries = (long long)htotal;
    // too many pairs for the caller's buffer, or for int32 cell offsets
    if ((long long)htotal > entry_cap || htotal >= 0x7fffffffull) return cudaSuccess;
    cell_count_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(rec, box_hi, nt, dims[0], dims[1], cnt);
    scan_reduce_kernel<<<(int)ntiles, SCAN_THREADS, 0, s>>>(cnt, nc, sums);
    scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(sums, ntiles);
    scan_final_kernel<<<(int)ntiles, SCAN_THREADS, 0, s>>>(cnt, nc, sums, cell_start);
    cell_fill_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(rec, box_hi, nt, dims[0], dims[1], cell_start, cursor,
                                                         tri_ids);
    cell_sort_kernel<<<blocks_for(nc, 256), 256, 0, s>>>(cell_start, nc, tri_ids);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *done = true;
    return cudaSuccess;
}
