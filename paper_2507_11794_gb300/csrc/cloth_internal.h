// Internal declarations shared by the translation units of libcloth.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cloth.h"

// Device-side control block of one cloth (one per handle, in device memory).
struct DevCtrl {
    unsigned long long k;     // global substep counter: selects time and ping-pong buffer
    unsigned int blocks_done; // completion counter of the running substep launch
    unsigned int flags;       // CTRL_FLAG_* (sticky until set_state)
    unsigned int coll_count;  // marked nodes of the running substep
    unsigned int pad;
    // running collision statistics since create: listed nodes, candidate
    // triangles tested, nodes that hit (summed over substeps)
    unsigned long long stat_listed, stat_tested, stat_hits;
};

// NONFINITE: a stored value was NaN/Inf; TIMEOUT: a bounded wait gave up;
// PARITY: a walk launched with a buffer parity that the substep counter
// contradicts (a host bookkeeping error; its results are wrong)
enum : unsigned int { CTRL_FLAG_NONFINITE = 1u, CTRL_FLAG_TIMEOUT = 2u, CTRL_FLAG_PARITY = 4u };

// Spring directions (drow, dcol) of the canonical order; each node owns the
// springs towards these six offsets ("forward"), and receives the other
// end of the springs of the six nodes at the negated offsets ("backward").
#define CLOTH_NDIR 6

// Everything one substep launch needs.  Plain data, passed by value.
struct StepParams {
    int nx, ny, n;
    int pitch;                 // floats per row (nx rounded up to 4): node (r,c) at r*pitch + c
    int rows_per_warp;         // rows walked by one warp
    int parity;                // walk launches: k & 1 as the host knows it when it enqueues the launch (the
                               // walk then picks its buffers without waiting for k), or -1: read k first
    int strips_x, strips_y;    // warp strips across columns / rows
    long long stride;          // floats between SoA planes
    float *state0, *state1;    // 6 planes each: px py pz vx vy vz
    const uint32_t *pin_bits;  // one bit per r*pitch + c, or nullptr
    const float *ks_slot;      // 6 planes [dir][r*pitch + c] (0 where no spring) or nullptr
    const float *kd_slot;
    float ks[3], kd[3];        // per type (used without per-spring arrays)
    float L0[CLOTH_NDIR];      // rest length per direction
    float inv_mass, dt;
    float g[3];
    float pin_vel[3];          // pinned nodes: x += dt pin_vel, v = pin_vel
    // wind: phase = omega*t + phase0 + col*kc + row*kr
    int has_wind;
    float w_amp, w_dir[3];
    // omega and phase0 in turns as 64-bit binary fractions: the time phase of
    // substep k is (w_turn_step k + w_turn0) mod 2^64, times 2 pi / 2^64
    unsigned long long w_turn_step, w_turn0;
    float w_kc, w_kr;
    const float2 *wind_rows;   // (sin, cos) of row*kr per row
    const float2 *wind_cols;   // (sin, cos) of col*kc per column
    // surface model
    int has_mesh;
    const float4 *tri;         // 3 float4 per triangle: (v0, lo.x) (e1, lo.y) (e2, lo.z)
    const int *cell_start;
    const int *tri_ids;
    const float4 *etri;        // per grid entry: its triangle's 3 records (no dependent load)
    float go[3];
    float ginv;
    int gd[3];
    float mlo[3], mhi[3];      // box of the mesh's vertices, padded by 1e-4 of its size (early out)
    int *coll_list;            // node offsets marked for the collision kernel (capacity N)
    int *coll_cloth;           // batch mode: cloth index of each entry (nullptr for one cloth)
    float *vstar;              // optional 3 planes: velocity after integration (adjoint recompute)
    float *cdata;              // optional 10 planes: per hit node m, r, g1 / K, g2 / K (adjoint recompute)
    uint32_t *cbits;           // with cdata: one bit per plane offset, set for the nodes that hit
    float4 *force;             // per-node force buffer of the atomic spring path, or nullptr
    float4 *edge_resp;         // edge narrow phase: per list entry (response position, hit flag), or nullptr
    float4 *edge_hit;          // edge narrow phase: per edge (kind * stride + owner) first hit point, hit count
    float4 *edge_more;         // edge narrow phase: CLOTH_EDGE_MORE planes of 3 x stride later hit points
    unsigned long long *edge_stamp; // edge narrow phase: per node, 1 + the substep it was last listed in
    unsigned *coll_count;      // entries in coll_list (reset by the collision kernel)
    int coll_blocks;           // CTAs of the collision kernel
    float delta, eps, tmin, restitution;
    DevCtrl *ctrl;
};

// Edge narrow phase: hit points stored per edge after its first (an edge
// with more hits is walked again by the gather pass).
#define CLOTH_EDGE_MORE 3

// CTAs per SM of the collision kernels (grid = SMs x this).
#ifndef CLOTH_COLL_CTAS_PER_SM
#define CLOTH_COLL_CTAS_PER_SM 2
#endif

// Launch one substep (reads state k&1, writes the other, advances ctrl->k).
cudaError_t launch_substep(const StepParams &p, cudaStream_t s);
// The two kernels of a substep separately (with a surface model, the walk
// leaves the counter to the collision kernel).  With p.force set, the "walk"
// is the atomic spring kernel followed by the per-node integration kernel.
cudaError_t launch_walk(const StepParams &p, cudaStream_t s);
cudaError_t launch_atomic_forces_and_integrate(const StepParams &p, cudaStream_t s);
// Per-vertex normals of the positions in `state` (planes px, py, pz) into
// out[nx*ny][3].
cudaError_t launch_normals(const float *state, long long stride, int nx, int ny, int pitch, float *out, int sms,
                           cudaStream_t s);
cudaError_t launch_collide(const StepParams &p, cudaStream_t s);

// A batch of cloths stepped by one persistent walk launch per substep.
struct BatchArgs {
    const StepParams *params;  // one per cloth (device)
    const int4 *items;         // (cloth, strip x, strip y, cost), longest first
    int n_items;
    unsigned *work;            // next item (re-armed by the last CTA)
    DevCtrl *ctrl;             // shared substep counter and flags
    int *coll_list, *coll_cloth;
    unsigned *coll_count;
    int walk_blocks, coll_blocks;
    int variant;               // BATCH_VAR_* shared by every cloth, or BATCH_VAR_MIXED
};
enum : int { BATCH_VAR_MESH = 1, BATCH_VAR_PER_SPRING = 2, BATCH_VAR_MIXED = 4 };
cudaError_t launch_batch_substep(const BatchArgs &b, cudaStream_t s);
int substep_strip_cols();
int substep_warps_per_cta();
int substep_min_ctas();
int batch_min_ctas();
// Longest walk of one warp (rows); the walk marks rows in 32-bit masks.
#define CLOTH_MAX_ROWS_PER_WARP 32
// Rows per warp of the column walk for a grid and SM count; strips from it.
int substep_rows_per_warp(int nx, int ny, int sm_count);
void substep_shape(StepParams &p);

// Grid over a surface model, built on the device.
struct DevGrid {
    float h, inv;
    float origin[3];
    int dims[3];
    long long ncells;
    long long nentries;
    float4 *tri;       // 3 per triangle
    int *cell_start;   // ncells + 1
    int *tri_ids;      // nentries
    float4 *etri;      // 3 per entry: copy of the entry's triangle record
    int ntris;
    float lo[3], hi[3];  // box of the triangles' vertices
};

// Host-side grid parameters (FP64 mean of the triangles' longest AABB side).
int grid_params(const float *verts, const int32_t *tris, int32_t nt, float *h, float origin[3], int dims[3],
                float *inv);

// Build the device grid from device copies of the mesh (d_verts, d_tris).
// Allocates g->tri, g->cell_start, g->tri_ids; scratch is allocated and
// freed inside.  Synchronises s.
cudaError_t grid_build(const float *d_verts, const int *d_tris, int ntris, DevGrid *g, cudaStream_t s);
void grid_free(DevGrid *g);

// Candidate query for debug/tests: counts[i], ids[i*cap..] (device arrays).
cudaError_t grid_query(const DevGrid &g, const float *dS, const float *dE, int nseg, int *counts, int *ids, int cap,
                       cudaStream_t s);

// AoS <-> SoA state transfer through the ping-pong buffer selected by ctrl->k.
cudaError_t launch_aos_to_soa(const float *aos_pos, const float *aos_vel, float *state0, float *state1,
                              long long stride, int n, int nx, int pitch, DevCtrl *ctrl, cudaStream_t s);
cudaError_t launch_soa_to_aos(const float *state0, const float *state1, long long stride, int n, int nx, int pitch,
                              const DevCtrl *ctrl, float *aos_pos, float *aos_vel, cudaStream_t s);

#ifdef __CUDACC__
// The wind's time phase omega k + phase0 reduced to [0, 2 pi), in float.
// omega and phase0 are held in turns as 64-bit binary fractions, so the
// reduction modulo one turn is the wrap of integer arithmetic: no FP64 on
// the device (a few FP64 operations cost this part more than the integer
// multiply).  Every kernel that needs the phase calls this, so they agree bit
// for bit.
__device__ __forceinline__ float wind_base(unsigned long long turn_step, unsigned long long turn0,
                                           unsigned long long k)
{
    const unsigned long long t = turn_step * k + turn0;         // turns, in units of 2^-64, mod 1
    return __uint2float_rn((unsigned)(t >> 32)) * 1.46291808e-9f;  // the top 32 bits times 2 pi / 2^32
}

// Grid cell coordinate of one float coordinate: floor((x - o) * inv) in
// float32, round-to-nearest with no contraction, clamped to [0, dim-1]
// (NaN -> 0).  Broad-phase candidate sets are defined by this formula, so it
// must stay exactly this sequence of rounded operations.
__device__ __forceinline__ int cell_coord(float x, float o, float inv, int dim)
{
    float f = floorf(__fmul_rn(__fsub_rn(x, o), inv));
    if (!(f >= 0.0f)) f = 0.0f;
    if (f > (float)(dim - 1)) f = (float)(dim - 1);
    return (int)f;
}
#endif

// Grid build into caller-supplied outputs and scratch (no allocation); see
// cloth_grid.cu.
cudaError_t grid_build_noalloc(const float *d_verts, const int *d_tris, int nt, const float origin[3], float inv,
                               const int dims[3], float4 *rec, int *cell_start, int *tri_ids, long long entry_cap,
                               int4 *box_hi, unsigned *cnt, unsigned *cursor, unsigned *sums,
                               unsigned long long *total, long long *nentries, bool *done, cudaStream_t s);

// Sets the calling thread's cloth_last_error() message.
void cloth_set_error_message(const char *msg);

// One cloth (the opaque handle of the C ABI).
struct ClothHandle {
    ClothDesc desc;  // array pointers cleared after the copy
    int n = 0;
    int pitch = 0;           // floats per row: nx rounded up to 4
    int sm_count = 0;
    long long stride = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    float *state = nullptr;  // 2 buffers x 6 planes x stride
    uint32_t *pin_bits = nullptr;
    float *ks_slot = nullptr, *kd_slot = nullptr;
    DevCtrl *ctrl = nullptr;
    float *staging = nullptr;  // 6*n floats for AoS transfers
    int *coll_list = nullptr;  // n entries
    float2 *wind_tab = nullptr; // ny row entries then nx column entries
    float4 *force = nullptr;    // CLOTH_FLAG_ATOMIC_SPRINGS: pitch*ny force accumulators
    float4 *edge_resp = nullptr; // CLOTH_FLAG_EDGE_COLLISION: n response slots (one per list entry)
    float4 *edge_hit = nullptr;      // CLOTH_FLAG_EDGE_COLLISION: 3 x stride edge records
    float4 *edge_more = nullptr;     // CLOTH_FLAG_EDGE_COLLISION: CLOTH_EDGE_MORE x 3 x stride hit points
    unsigned long long *edge_stamp = nullptr;  // CLOTH_FLAG_EDGE_COLLISION: stride listing stamps
    DevGrid grid{};
    bool has_mesh = false;
    StepParams params{};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one step, by the parity of its first substep
    unsigned long long params_gen = 0;  // bumped by cloth_fill_params: graphs built from older params are stale
    long long substeps_done = 0;
    bool dead = false;
};

void cloth_fill_params(ClothHandle *h);
