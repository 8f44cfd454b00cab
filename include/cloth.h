/*
 * cloth.h -- C ABI of the GB300 mass-spring cloth library (libcloth.so).
 *
 * The library steps the per-timestep hot path of the mass-spring cloth of
 * "Real-Time Cloth Simulation Using WebGPU" (arXiv 2507.11794) on one GPU:
 *   - spring + damping forces of the structural, shear and bend springs of a
 *     grid cloth (Section 3 "Methodology"; Algorithm 1, Hooke's law with
 *     damping along the spring), gathered per node in a fixed order;
 *   - "the Euler method" with spring force, gravity and external force
 *     (Section 3), read as symplectic Euler, with pinned nodes (the hanging
 *     cloth of Section 4.1);
 *   - collision with a static ("baked", Section 4.2) triangle surface model:
 *     a uniform-grid broad phase (not in the paper, which tests all pairs) and
 *     the extended Moller-Trumbore test on each node's substep path
 *     (Section 3, "Extended Moller-Trumbore Process");
 *   - the collision response of Section 3 and Algorithm 2: on K > 0 hits the
 *     node restarts from its previous position plus the average response
 *     (1/K) sum_k max(t_k - delta, 0) * r, and its velocity is scaled by
 *     `restitution` (Algorithm 2: -0.5).
 *
 * Conventions
 *   - Every call returns 0 (CLOTH_OK) or a negative CLOTH_ERR_* code; nothing
 *     throws across the ABI.  cloth_last_error() returns a message for the
 *     calling thread's most recent failure.
 *   - Ownership: the library owns all device memory it allocates; callers own
 *     every host buffer they pass, which is only read during the call.
 *   - Layout of host node arrays: N = nx*ny nodes, node id = row*nx + col;
 *     positions and velocities are AoS float32 [N][3].
 *   - Streams: all GPU work of a handle runs on the stream given at create
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *     cloth_step is asynchronous; cloth_read and cloth_sync synchronise the
 *     stream.  Errors raised by earlier asynchronous work (a non-finite
 *     state, a CUDA fault) are reported by the next synchronising call.
 *   - After CLOTH_ERR_CUDA a handle is unusable: every call but
 *     cloth_destroy returns CLOTH_ERR_STATE.
 *   - Handles are not thread-safe; distinct handles may be used from
 *     distinct threads.
 */
#ifndef CLOTH_H
#define CLOTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CLOTH_OK = 0,
    CLOTH_ERR_INVALID_ARG = -1, /* bad pointer, size or parameter */
    CLOTH_ERR_OOM = -2,         /* device or host allocation failed */
    CLOTH_ERR_CUDA = -3,        /* a CUDA call failed; the handle is now unusable */
    CLOTH_ERR_NONFINITE = -4,   /* a position or velocity became NaN/Inf */
    CLOTH_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    CLOTH_ERR_BAD_MESH = -6,    /* triangle index out of range, bad sizes */
    CLOTH_ERR_STATE = -7        /* handle unusable after an earlier CUDA error */
};

/* Flags of ClothDesc.flags */
#define CLOTH_FLAG_NO_GRAPH 1u /* launch substeps one by one instead of a CUDA graph */
/* Evaluate the spring forces as Algorithm 1 prints them: one thread per
 * spring adding F to one end and -F to the other with FP32 atomic adds into a
 * per-node force buffer (16 B per node, zeroed again by the integration kernel
 * as Algorithm 2 resets its buffers), then one thread per node integrating.
 * The force law, integrator and collision phase are those of the default
 * path, but the order of the additions, and so the last bits of the state,
 * vary from run to run.  Kept as an A/B of the paper's design against the
 * default fused column walk.  Not accepted by cloth_batch_create or
 * cloth_rollout_create (the adjoint recomputes segments and needs bitwise
 * reproducible forward states). */
#define CLOTH_FLAG_ATOMIC_SPRINGS 2u
/* The paper's own narrow phase instead of the node-path test: the edges of
 * the cloth triangles (the grid's quads split along their (r,c)-(r+1,c+1)
 * diagonal) at the updated positions are tested against the surface
 * triangles with the extended Moller-Trumbore test (Section 3); every vertex
 * of the cloth triangles sharing a hit edge moves from its previous position
 * towards the hit point, stopping contact_offset short, averaged over its
 * hits, and its velocity is scaled by restitution (Algorithm 2).  A
 * separate pass lists every node whose neighbourhood (its 3 x 3 block of
 * nodes at the updated positions) has a box overlapping the mesh's grid, which
 * holds every node of a triangle with an edge that can hit, however far the
 * cloth is stretched.  Edges parallel to the surface are not detected (the
 * test's parallel rule).  Not accepted by cloth_batch_create or
 * cloth_rollout_create. */
#define CLOTH_FLAG_EDGE_COLLISION 4u

/* Sinusoidal external acceleration field (N/kg) added to gravity:
 *   w(X0, t) = amp * dir * sin(2*pi*freq*t + kappa*(udir . X0) + phase),
 * X0 the node's rest position, t = k*dt_s the start time of substep k.
 * amp = 0 disables it. */
typedef struct ClothWind {
    float amp;
    float dir[3];
    float udir[3];
    float freq;
    float kappa;
    float phase;
} ClothWind;

/* Problem statement of one cloth (caller-owned; copied by cloth_create).
 * The paper's inputs: springs with stiffness, rest length and damping
 * (Algorithm 1), node positions/velocities (Algorithm 2), masses, gravity,
 * external force and the Euler time step (Section 3). */
typedef struct ClothDesc {
    int32_t nx, ny;          /* grid resolution in nodes (>= 1 each); N = nx*ny */
    float origin[3];         /* rest position of node (0,0) */
    float du[3], dv[3];      /* rest offsets between columns / rows:
                                X0(row,col) = origin + col*du + row*dv; rest
                                lengths come from this flat grid */
    float total_mass;        /* kg, spread uniformly: m = total_mass / N */
    float ks[3], kd[3];      /* per type (structural, shear, bend): N/m, N*s/m */
    const float *ks_spring;  /* optional host array of S floats in canonical
                                spring order (below), overriding ks[]; NULL = off */
    const float *kd_spring;  /* optional, likewise for kd */
    const float *init_pos;   /* optional host [N][3]; NULL = the flat grid X0 */
    const float *init_vel;   /* optional host [N][3]; NULL = 0 */
    const uint8_t *pinned;   /* optional host [N], nonzero = pinned; NULL = none */
    float gravity[3];        /* m/s^2 */
    float dt;                /* time advanced by one cloth_step (s) */
    int32_t substeps;        /* substeps per cloth_step (>= 1); dt_s = dt/substeps */
    float contact_offset;    /* delta (m): a hit stops the node delta before it */
    float mt_eps;            /* epsilon of the extended MT parallel test |a| < eps */
    float mt_t_min;          /* hits need mt_t_min < t < |d| (paper text: eps) */
    float restitution;       /* velocity factor on contact (Algorithm 2: -0.5) */
    ClothWind wind;
    uint32_t flags;          /* CLOTH_FLAG_* */
    float pin_velocity[3];   /* m/s: pinned nodes move kinematically,
                                x += dt_s*pin_velocity, v = pin_velocity (the
                                paper's pulling scene); 0 = fixed pins */
} ClothDesc;

/* Canonical spring order (for ks_spring / kd_spring): nodes in row-major
 * order, each emitting its springs towards (drow,dcol) = (0,+1), (+1,0),
 * (+1,+1), (+1,-1), (0,+2), (+2,0) when the other end lies in the grid.
 * Types: the first two structural, the next two shear, the last two bend.
 * S = 2*nx*ny - nx - ny + 2*(nx-1)*(ny-1) + nx*(ny-2)^+ + ny*(nx-2)^+. */

typedef struct ClothHandle ClothHandle;

/* Create a cloth on the current CUDA device.  desc is validated (sizes,
 * finiteness, dt > 0, substeps >= 1, total_mass > 0) and copied with its
 * arrays; stream is the cudaStream_t all work of the handle runs on.
 * Returns CLOTH_ERR_INVALID_ARG, CLOTH_ERR_OOM or CLOTH_ERR_CUDA on failure
 * (*out is then NULL). */
int cloth_create(const ClothDesc *desc, void *stream, ClothHandle **out);

/* Set (or with ntris = 0 clear) the static surface model: host arrays of
 * nverts*3 float32 vertex coordinates and ntris*3 int32 vertex indices,
 * copied.  Builds the uniform grid on the device (counting sort of the
 * (cell, triangle) pairs).  Indices outside [0, nverts) or non-finite
 * vertices return CLOTH_ERR_BAD_MESH and leave the previous mesh in place.
 * Synchronises the stream. */
int cloth_set_mesh(ClothHandle *h, const float *verts, int32_t nverts, const int32_t *tris, int32_t ntris);

/* Enqueue nsteps steps (nsteps * substeps substeps) on the stream.  Each
 * substep: spring and damping forces (Algorithm 1), symplectic Euler with
 * gravity, wind and pins (Section 3), then, with a surface model, the grid
 * broad phase, the extended Moller-Trumbore narrow phase and the averaged
 * response (Algorithm 2).  Replayed from a CUDA graph of one step unless
 * CLOTH_FLAG_NO_GRAPH.  Errors: CLOTH_ERR_INVALID_ARG (nsteps < 0),
 * CLOTH_ERR_CUDA; device-side flags are reported by the next cloth_sync or
 * cloth_read. */
int cloth_step(ClothHandle *h, int32_t nsteps);

/* Copy the current state to caller-owned host [N][3] arrays (either may be
 * NULL).  Synchronises; returns CLOTH_ERR_NONFINITE if the state has become
 * non-finite since create/set_state (the arrays are still written). */
int cloth_read(ClothHandle *h, float *pos_out, float *vel_out);

/* Release everything the handle owns.  NULL-safe.  Synchronises the stream. */
void cloth_destroy(ClothHandle *h);

/* ---- extras --------------------------------------------------------- */

/* Overwrite the current state from host [N][3] arrays (NULL keeps that
 * part) and clear the non-finite flag.  Asynchronous for pinned host memory
 * (the host arrays must stay valid until the stream reaches the copy);
 * pageable memory is copied before return. */
int cloth_set_state(ClothHandle *h, const float *pos, const float *vel);

/* Wait for the handle's stream and report device-side error flags. */
int cloth_sync(ClothHandle *h);

/* Running totals of the collision phase since create, summed over substeps
 * (not part of the paper, which gives no counts; they describe the work of
 * the grid broad phase and narrow phase of Section 3): listed = nodes whose
 * substep path box reached the surface model's (padded) bounding box,
 * tested = candidate triangles put through the extended Moller-Trumbore
 * test, hits = nodes that received a response.  With the edge narrow phase
 * (CLOTH_FLAG_EDGE_COLLISION): listed = nodes whose 3 x 3 block box reached
 * that box, tested = candidate triangles of their owned edges, hits = edges
 * with at least one hit.  Zero without a surface model.  Synchronises.  Any
 * output may be NULL.  Errors: CLOTH_ERR_INVALID_ARG, CLOTH_ERR_STATE,
 * CLOTH_ERR_CUDA. */
int cloth_get_collision_stats(ClothHandle *h, int64_t *listed, int64_t *tested, int64_t *hits);

/* Thread-local message of the last failed call ("" if none). */
const char *cloth_last_error(void);

typedef struct ClothInfo {
    int32_t nx, ny, n;
    int32_t substeps;
    int64_t substeps_done;     /* substeps enqueued since create */
    int64_t plane_stride;      /* floats between consecutive SoA planes */
    float *pos_planes[3];      /* device pointers of the current x,y,z planes: node */
    float *vel_planes[3];      /* (row,col) at [row*row_pitch + col]; valid once the
                                  enqueued work has run, until the next step/set_state */
    int32_t ntris;
    int32_t grid_dims[3];
    float grid_origin[3];
    float grid_h, grid_inv;
    int64_t grid_entries;
    int32_t has_per_spring;
    int32_t row_pitch;         /* floats per row in the SoA planes (nx rounded up to 4) */
} ClothInfo;

/* Sizes, grid parameters and device pointers of the current SoA state. */
int cloth_get_info(ClothHandle *h, ClothInfo *info);

/* Copy the uniform grid to host arrays: cell_start [cells+1] and tri_ids
 * [grid_entries] (each cell's ids ascending).  Synchronises. */
int cloth_get_grid(ClothHandle *h, int32_t *cell_start, int32_t *tri_ids);

/* Broad-phase query on the device for nseg float32 segments S->E (host
 * [nseg][3] arrays): counts[i] = number of distinct candidate triangles of
 * segment i (the triangles listed in the grid cells overlapped by the
 * segment's AABB); ids receives up to cap ids per segment at ids[i*cap ..],
 * in no particular order.  Synchronises. */
int cloth_query_candidates(ClothHandle *h, const float *S, const float *E, int32_t nseg,
                           int32_t *counts, int32_t *ids, int32_t cap);

/* Advance nsub substeps with every kernel launch bracketed by CUDA events
 * (captured into a graph and replayed once on the handle's stream, so the
 * launches run back to back), and report the mean device
 * duration per launch in microseconds: walk_us for the force + integration
 * kernel (Algorithm 1 and Section 3), collide_us for the collision kernel
 * (Section 3 and Algorithm 2; 0 without a surface model).  The state
 * advances exactly as with cloth_step.  nsub in [1, 4096]; either output may
 * be NULL.  Synchronises.  Errors: CLOTH_ERR_INVALID_ARG, CLOTH_ERR_CUDA,
 * and the flag errors of cloth_sync. */
int cloth_profile_substeps(ClothHandle *h, int32_t nsub, float *walk_us, float *collide_us);

/* Per-vertex normals of the current positions: the normal update that ends
 * a frame before rendering (Section 3), computed headless.  Each grid quad is
 * split along its (r,c)-(r+1,c+1) diagonal; a vertex normal is the normalised
 * sum of the unnormalised face normals of the (up to six) triangles
 * containing the vertex, the zero vector where that sum is zero.
 * d_normals: DEVICE pointer to nx*ny*3 floats (node-major, x y z), owned by
 * the caller; written asynchronously on the handle's stream, after the
 * substeps already queued.  Errors: CLOTH_ERR_INVALID_ARG (NULL), CLOTH_ERR_CUDA. */
int cloth_compute_normals(ClothHandle *h, float *d_normals);

/* ---- batches of cloths ------------------------------------------------- */

/* Many independent cloths (each with its own grid, constants, pins and
 * surface model) stepped together: every substep is one persistent walk
 * launch over a (cloth, strip) work list sorted longest first plus one
 * collision launch over the nodes of all cloths near their meshes, replayed
 * from a CUDA graph holding one step.  Each cloth gets exactly the arithmetic
 * it gets from cloth_step (bitwise the same results).  Not in the paper. */
typedef struct ClothBatch ClothBatch;

typedef struct ClothBatchTuning {
    int32_t rows_per_warp;     /* strip height of one warp's walk */
    int32_t walk_ctas_per_sm;  /* persistent walk grid = SMs x this */
    float us_per_substep;      /* measured by cloth_batch_tune (0 otherwise) */
    int32_t candidates;        /* configurations timed by cloth_batch_tune */
} ClothBatchTuning;

/* count descriptions (all with the same dt and substeps), each validated and
 * copied as by cloth_create; all work runs on stream. */
int cloth_batch_create(const ClothDesc *descs, int32_t count, void *stream, ClothBatch **out);
/* cloth_set_mesh for cloth `index` of the batch.  Synchronises. */
int cloth_batch_set_mesh(ClothBatch *b, int32_t index, const float *verts, int32_t nverts, const int32_t *tris,
                         int32_t ntris);
/* Enqueue nsteps steps of every cloth. */
int cloth_batch_step(ClothBatch *b, int32_t nsteps);
/* cloth_read for cloth `index`.  Synchronises; CLOTH_ERR_NONFINITE if any
 * cloth of the batch became non-finite. */
int cloth_batch_read(ClothBatch *b, int32_t index, float *pos_out, float *vel_out);
/* cloth_set_state for cloth `index` (clears the batch's non-finite flag). */
int cloth_batch_set_state(ClothBatch *b, int32_t index, const float *pos, const float *vel);
/* Autotuner: times trial_substeps substeps of the batch for every candidate
 * (rows_per_warp in {4,6,8,12,16,24,32} x walk CTAs per SM), keeps the
 * fastest, and restores every cloth's state and the substep counter, so the
 * simulation is unchanged.  Synchronises. */
int cloth_batch_tune(ClothBatch *b, int32_t trial_substeps, ClothBatchTuning *out);
/* Set the tuning explicitly (rows_per_warp 1..32, walk_ctas_per_sm 1..32). */
int cloth_batch_set_tuning(ClothBatch *b, int32_t rows_per_warp, int32_t walk_ctas_per_sm);
int cloth_batch_get_tuning(ClothBatch *b, ClothBatchTuning *out);
/* Wait for the batch's stream and report device-side error flags. */
int cloth_batch_sync(ClothBatch *b);
/* Running collision totals of the whole batch since create, summed over its
 * cloths and substeps, as cloth_get_collision_stats gives them for one
 * cloth.  Synchronises.  Any output may be NULL.  Errors:
 * CLOTH_ERR_INVALID_ARG, CLOTH_ERR_STATE, CLOTH_ERR_CUDA. */
int cloth_batch_get_collision_stats(ClothBatch *b, int64_t *listed, int64_t *tested, int64_t *hits);
/* Release the batch and its cloths.  NULL-safe. */
void cloth_batch_destroy(ClothBatch *b);

/* ---- differentiation --------------------------------------------------- */

/* A rollout of nsteps steps of one cloth with its reverse pass (not in the
 * paper): the gradient of a loss on the final state w.r.t. every spring's
 * stiffness and damping (canonical spring order) and the initial
 * velocities.  The contact set of every substep is frozen at the one the
 * forward pass finds (the response is differentiated as a smooth map of the
 * start point and the path direction).  The forward pass stores the state
 * every checkpoint_every steps; the backward pass recomputes one segment at
 * a time into one of two slot sets while the previous segment is reversed,
 * so device memory grows as nsteps/checkpoint_every states plus
 * 2 x (checkpoint_every x substeps + 1) slots of 19 planes.  The forward and
 * backward passes run as CUDA graphs captured on first use (rebuilt after
 * cloth_set_mesh) unless the cloth has CLOTH_FLAG_NO_GRAPH; the backward
 * pass also uses a stream of the rollout's own, joined to the cloth's stream
 * before the call's last work.  All pointers below are device pointers on
 * the cloth's device; all calls run on the cloth's stream. */
typedef struct ClothRollout ClothRollout;

/* The cloth's current state (at its current substep count) becomes the
 * rollout's initial state.  A cloth created without per-spring constants gets
 * per-spring planes filled from its per-type constants.  Errors:
 * CLOTH_ERR_INVALID_ARG (NULL, nsteps or checkpoint_every < 1, a cloth created
 * with CLOTH_FLAG_ATOMIC_SPRINGS or CLOTH_FLAG_EDGE_COLLISION), CLOTH_ERR_OOM,
 * CLOTH_ERR_CUDA. */
int cloth_rollout_create(ClothHandle *h, int32_t nsteps, int32_t checkpoint_every, ClothRollout **out);
/* Forward pass from the initial state: d_ks, d_kd (S floats, canonical
 * order; NULL keeps the current constants), d_v0 ([N][3] initial velocities;
 * NULL = the initial state's).  Writes the final state to d_pos_out /
 * d_vel_out ([N][3], either may be NULL); the cloth then holds that state. */
int cloth_rollout_forward(ClothRollout *ro, const float *d_ks, const float *d_kd, const float *d_v0, float *d_pos_out,
                          float *d_vel_out);
/* Reverse pass of the last forward: d_gpos, d_gvel = dL/d(final positions,
 * velocities) ([N][3]; d_gvel may be NULL = 0).  Writes dL/dks, dL/dkd (S
 * floats) and dL/dv0 ([N][3]); any output may be NULL.  The cloth is left in
 * the final forward state. */
int cloth_rollout_backward(ClothRollout *ro, const float *d_gpos, const float *d_gvel, float *d_gks, float *d_gkd,
                           float *d_gv0);
/* NULL-safe; the cloth itself stays alive. */
void cloth_rollout_destroy(ClothRollout *ro);

/* ---- allocation-free grid build --------------------------------------- */

/* Largest mesh and grid cloth_grid_build_static accepts. */
#define CLOTH_STATIC_GRID_MAX_TRIS 131072
#define CLOTH_STATIC_GRID_MAX_VERTS 131072
#define CLOTH_STATIC_GRID_MAX_CELLS 262144

typedef struct ClothGridParams {
    float h, inv;       /* cell size and its float reciprocal */
    float origin[3];    /* corner of cell (0,0,0) */
    int32_t dims[3];    /* cells per axis; cell id = (z*dims[1] + y)*dims[0] + x */
    int64_t ncells;     /* dims[0]*dims[1]*dims[2] */
    int64_t nentries;   /* (cell, triangle) pairs = length of tri_ids; -1 if not counted */
} ClothGridParams;

/* The paper has no counterpart to this entry point: it is a variant of the
 * grid build inside cloth_set_mesh for callers that must not allocate device
 * memory -- hosts that run under an allocator with a fixed budget, or that
 * forbid cudaMalloc/cudaFree once start-up is over.  It calls no allocating
 * routine: its temporaries live in one fixed-size device array of the library
 * (7,341,312 bytes), and the caller supplies the outputs.  A device holds that
 * array from the moment the library's module is loaded on it until the
 * process exits; with CUDA's lazy module loading (the default) the load can
 * happen at the first call on that device, so a caller that may not allocate
 * later makes one call per device during start-up.
 *
 * Inputs: host arrays verts [nverts][3] float32 and tris [ntris][3] int32
 * (the same mesh cloth_set_mesh takes), at most CLOTH_STATIC_GRID_MAX_TRIS
 * triangles, CLOTH_STATIC_GRID_MAX_VERTS vertices and a grid of at most
 * CLOTH_STATIC_GRID_MAX_CELLS cells; larger inputs are rejected with
 * CLOTH_ERR_INVALID_ARG before any GPU work.  stream: the cudaStream_t to run
 * on (NULL = legacy default stream); the call synchronises it.
 * Outputs (caller-owned device memory of the current device):
 *   d_tri_records  12*ntris floats, 16-byte aligned: per triangle the float4s
 *                  (v0, lo.x) (v1-v0, lo.y) (v2-v0, lo.z), lo = first cell;
 *   d_cell_start   cell_capacity >= ncells+1 ints (exclusive prefix of counts);
 *   d_tri_ids      entry_capacity >= nentries ints, each cell's ids ascending.
 * params receives the grid parameters, nentries once counted.  If a capacity
 * is too small the call returns CLOTH_ERR_INVALID_ARG with params filled as
 * far as known (ncells always, nentries when the cells fitted), so a caller
 * can size its buffers with calls of zero capacity.  The results are
 * identical to the grid cloth_set_mesh builds for the same mesh.
 *
 * Every call shares the one scratch array and leaves its last contents
 * there; each call clears what must start at zero.  Calls whose GPU work
 * overlaps (on different streams, or from different threads on the same
 * device) race on the scratch and give wrong results: serialise them.  The
 * first call on each device looks the array's device address up (with that
 * device current); with lazy module loading that first call may load the
 * library's module and allocate the array then.
 * Errors: CLOTH_ERR_INVALID_ARG (limits, capacities, a device index of 64 or
 * more), CLOTH_ERR_BAD_MESH (index out of range, non-finite vertex, 2^31 - 1
 * or more (cell, triangle) pairs), CLOTH_ERR_CUDA. */
int cloth_grid_build_static(const float *verts, int32_t nverts, const int32_t *tris, int32_t ntris, void *stream,
                            float *d_tri_records, int32_t *d_cell_start, int64_t cell_capacity,
                            int32_t *d_tri_ids, int64_t entry_capacity, ClothGridParams *params);

#ifdef __cplusplus
}
#endif

#endif /* CLOTH_H */
