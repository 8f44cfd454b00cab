// One substep of the mass-spring cloth, fused into a single kernel:
//   spring + damping forces (Algorithm 1's force law, each spring evaluated
//   once), symplectic Euler with gravity, wind and pins (Section 3),
//   uniform-grid broad phase + extended Moller-Trumbore narrow phase on the
//   node's substep path (Section 3) and the averaged response of Algorithm 2.
//
// Layout: six SoA float planes (px py pz vx vy vz) per ping-pong buffer, rows
// of `pitch` floats (nx rounded up to 4); the launch reads buffer k&1 and
// writes the other, k = the device substep counter.
//
// Work decomposition (register-window column walk): each lane owns two
// adjacent columns (A = even, B = odd) held as float2 pairs, so every
// arithmetic instruction of the spring law works on both nodes at once
// (packed FP32x2).  A warp covers 64 columns, of which lanes 1..30 produce
// output (60 columns) and lanes 0 and 31 are the halo that bend springs need.
// The warp walks down `rows_per_warp` rows keeping rows r, r+1, r+2 in
// registers; neighbour data moves between lanes by shuffles.  Each node
// evaluates only its six "forward" springs (towards (0,+1), (0,+2), (+1,0),
// (+2,0), (+1,+1), (+1,-1)); the reaction -F of Algorithm 1 reaches the other
// end by shuffle (same row) or is carried in registers to the next rows.  So
// every spring is evaluated once, with no atomics and a fixed summation order:
// results are bitwise reproducible.  The first two rows of each walk only
// produce the springs that reach into the strip.
#include <type_traits>
#include <utility>

#include "cloth_collide.cuh"
#include "cloth_internal.h"

namespace {

// Tuning knobs of the walk kernel (defaults chosen by measurement):
// CTAs per SM the register budget targets, and the unroll of the row walk.
#ifndef CLOTH_WALK_MINB
#define CLOTH_WALK_MINB 12
#endif
#ifndef CLOTH_WALK_UNROLL
#define CLOTH_WALK_UNROLL 1
#endif
#ifndef CLOTH_COLL_MINB
#define CLOTH_COLL_MINB 2
#endif
#define CLOTH_PRAGMA(x) _Pragma(#x)
#define CLOTH_UNROLL(n) CLOTH_PRAGMA(unroll n)

constexpr unsigned FULL = 0xffffffffu;

// Programmatic dependent launch: each kernel of a substep lets the next one
// be launched once all its CTAs are running (launch_dependents), and waits
// for the previous one to complete, with its writes visible, before it
// touches any state (wait).  The next kernel's launch and CTA start-up then
// overlap this kernel's tail instead of following it.
#ifndef CLOTH_PDL
#define CLOTH_PDL 1
#endif
// Substep completion: the last CTA of the kernel that ends a substep (found by
// an atomic count of finished CTAs) advances the substep counter and resets
// the per-substep counters.  It reads nothing the other CTAs wrote, and every
// CTA has read those control words before its increment; the next kernel
// reads them only after this one has completed (or after griddepcontrol.wait),
// which makes all writes visible.  So no memory fence is taken: a fence would
// make each CTA wait for its own stores to drain, about 1 us per launch.
__device__ __forceinline__ void pdl_wait()
{
#if CLOTH_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_launch_dependents()
{
#if CLOTH_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
// One warp per CTA: the walk's warps fill one wave, and with 4-warp CTAs
// 403 CTAs of the 800 x 800 walk put 12 warps on two thirds of the SMs and 8
// on the rest, so the crowded SMs set the time; single-warp CTAs spread 10
// or 11 warps on every SM (11% faster without a mesh, 15% on the batch).
#ifndef CLOTH_WALK_WARPS
#define CLOTH_WALK_WARPS 1
#endif
constexpr int WARPS_PER_CTA = CLOTH_WALK_WARPS;
// register budget of the walk kernels: CLOTH_WALK_MAXREG registers per thread
// when given, else what CLOTH_WALK_MINB resident CTAs per SM leave
#ifdef CLOTH_WALK_MAXREG
#define CLOTH_WALK_BOUNDS __maxnreg__(CLOTH_WALK_MAXREG)
#else
#define CLOTH_WALK_BOUNDS __launch_bounds__(32 * CLOTH_WALK_WARPS, CLOTH_WALK_MINB)
#endif
// the batch kernel (its walk also stages each item's parameters) keeps its own
#ifndef CLOTH_BATCH_MINB
#define CLOTH_BATCH_MINB 12
#endif
constexpr int STRIP_COLS = 60;

// Packed FP32x2 arithmetic as explicitly rounded PTX instructions (add.rn,
// mul.rn, fma.rn on .f32x2).  Each is one IEEE operation per component that
// no optimizer fuses or reorders, so a node's arithmetic is the same whichever
// copy of the unrolled row loop computes it; with the CUDA 13.0 packed
// intrinsics (__fadd2_rn, __fmul2_rn, __ffma2_rn) the four copies of the loop
// gave results one ulp apart, so a cloth's bits depended on its strip height.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 x, y, d;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tadd.rn.f32x2 d, x, y;\n\t"
        "mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 x, y, d;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tmul.rn.f32x2 d, x, y;\n\t"
        "mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{.reg .b64 x, y, z, d;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tmov.b64 z, {%6, %7};\n\t"
        "fma.rn.f32x2 d, x, y, z;\n\tmov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
// a - b, exact as one rounding: fma(b, -1, a)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }

struct Node2 {  // two nodes (A = .x, B = .y)
    float2 px, py, pz, vx, vy, vz;
};
struct Vec2 {  // one 3-vector per node of the pair
    float2 x, y, z;
};

__device__ __forceinline__ Vec2 vadd(Vec2 a, Vec2 b) { return {add2(a.x, b.x), add2(a.y, b.y), add2(a.z, b.z)}; }
__device__ __forceinline__ Vec2 vsub(Vec2 a, Vec2 b) { return {sub2(a.x, b.x), sub2(a.y, b.y), sub2(a.z, b.z)}; }

__device__ __forceinline__ float2 shfl_down2(float2 v, int d)
{
    return make_float2(__shfl_down_sync(FULL, v.x, d), __shfl_down_sync(FULL, v.y, d));
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int d)
{
    return make_float2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
}
// Row r of the lane's two columns.  The row and the column pair are clamped
// into the grid's memory, so every load is in bounds; the values of a row
// outside [0, ny) or a pair outside the pitch are finite stand-ins that only
// enter springs whose constants are zero (no spring there).  Plane j of the
// buffer starts at in + j * st (32-bit offsets: creation keeps 6 st below
// 2^32).
__device__ __forceinline__ Node2 load_row(const float *in, unsigned st, int r, int ny, int pitch, int cmem)
{
    const int rr = min(max(r, 0), ny - 1);
    const unsigned o = (unsigned)rr * (unsigned)pitch + (unsigned)cmem;
    Node2 n;
    n.px = __ldg((const float2 *)(in + o));
    n.py = __ldg((const float2 *)(in + (o + st)));
    n.pz = __ldg((const float2 *)(in + (o + 2u * st)));
    n.vx = __ldg((const float2 *)(in + (o + 3u * st)));
    n.vy = __ldg((const float2 *)(in + (o + 4u * st)));
    n.vz = __ldg((const float2 *)(in + (o + 5u * st)));
    return n;
}

// Hooke's law plus damping along the spring (Algorithm 1) for the pair:
// d = q - p, F_p = (ks (|d| - L0) + kd (v_q - v_p).d / |d|) d / |d|, written
// as F_p = s d with s = (ks (|d| - L0) + kd il (v_q - v_p).d) il, il = 1/|d|
// (zero force for |d|^2 <= 1e-24).
// The same from the differences d = q - p (dx, dy, dz) and v_q - v_p (ux,
// uy, uz).
__device__ __forceinline__ Vec2 spring2d(float2 dx, float2 dy, float2 dz, float2 ux, float2 uy, float2 uz, float2 ks,
                                         float2 kd, float L0)
{
    const float2 l2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float2 il;
    il.x = l2.x > 1e-24f ? rsqrtf(l2.x) : 0.0f;
    il.y = l2.y > 1e-24f ? rsqrtf(l2.y) : 0.0f;
    const float2 dvd = fma2(uz, dz, fma2(uy, dy, mul2(ux, dx)));
    const float2 e = fma2(l2, il, bc(-L0));  // |d| - L0
    const float2 sc = mul2(fma2(mul2(kd, il), dvd, mul2(ks, e)), il);
    return {mul2(sc, dx), mul2(sc, dy), mul2(sc, dz)};
}
__device__ __forceinline__ Vec2 spring2(const Node2 &P, const Node2 &Q, float2 ks, float2 kd, float L0)
{
    return spring2d(sub2(Q.px, P.px), sub2(Q.py, P.py), sub2(Q.pz, P.pz), sub2(Q.vx, P.vx), sub2(Q.vy, P.vy),
                    sub2(Q.vz, P.vz), ks, kd, L0);
}
// A spring of each node of the pair P towards the pair Q = (a.y, b.x) that
// straddles two column pairs: the differences are formed one component at a
// time, so Q is never assembled.
__device__ __forceinline__ float2 dstr(float ay, float bx, float2 p) { return make_float2(__fsub_rn(ay, p.x), __fsub_rn(bx, p.y)); }
__device__ __forceinline__ Vec2 spring2s(const Node2 &P, const Node2 &a, const Node2 &b, float2 ks, float2 kd,
                                         float L0)
{
    return spring2d(dstr(a.px.y, b.px.x, P.px), dstr(a.py.y, b.py.x, P.py), dstr(a.pz.y, b.pz.x, P.pz),
                    dstr(a.vx.y, b.vx.x, P.vx), dstr(a.vy.y, b.vy.x, P.vy), dstr(a.vz.y, b.vz.x, P.vz), ks, kd, L0);
}

// Sign bits set (node A in .x, node B in .y) where the segment from s to e
// lies on the far side of one face of the slab [lo, hi]: both ends below lo
// or both above hi.
__device__ __forceinline__ uint2 box_out_bits(float2 s, float2 e, float lo, float hi)
{
    const float2 a = sub2(s, bc(lo)), b = sub2(e, bc(lo)), c = sub2(bc(hi), s), d = sub2(bc(hi), e);
    return make_uint2((__float_as_uint(a.x) & __float_as_uint(b.x)) | (__float_as_uint(c.x) & __float_as_uint(d.x)),
                      (__float_as_uint(a.y) & __float_as_uint(b.y)) | (__float_as_uint(c.y) & __float_as_uint(d.y)));
}

// q - (ay, bx) for a pair q and the straddling pair (a.y, b.x), one
// component at a time.
__device__ __forceinline__ float2 rdstr(float2 q, float ay, float bx) { return make_float2(__fsub_rn(q.x, ay), __fsub_rn(q.y, bx)); }
__device__ __forceinline__ Vec2 vscale(Vec2 a, float2 s) { return {mul2(a.x, s), mul2(a.y, s), mul2(a.z, s)}; }


// Inputs of a strip that do not change from substep to substep (the wind
// tables and the pin bits): the lane's column wind terms and the first output
// row's entries.  The single-cloth kernel loads them before it waits for the
// previous substep, so their latency hides behind that wait.
struct WalkStatics {
    float2 sinB, cosB;  // (sin, cos) of the column phase of the lane's two columns
    float2 trN;         // (sin, cos) of row r0's phase
    unsigned pinN;      // the pin word holding row r0's bit of the lane's column A
};

__device__ __forceinline__ WalkStatics walk_statics(const StepParams &p, int sx, int sy, int lane)
{
    WalkStatics w;
    const int cA = sx * STRIP_COLS - 2 + 2 * lane;
    const int r0 = sy * p.rows_per_warp;
    w.sinB = w.cosB = make_float2(0.0f, 0.0f);
    w.trN = make_float2(0.0f, 1.0f);
    w.pinN = 0u;
    if (p.has_wind) {
        if (cA >= 0 && cA < p.nx) {
            const float2 t = __ldg(p.wind_cols + cA);
            w.sinB.x = t.x;
            w.cosB.x = t.y;
        }
        if (cA + 1 >= 0 && cA + 1 < p.nx) {
            const float2 t = __ldg(p.wind_cols + cA + 1);
            w.sinB.y = t.x;
            w.cosB.y = t.y;
        }
        if (r0 < p.ny) w.trN = __ldg(p.wind_rows + r0);
    }
    if (p.pin_bits && cA >= 0 && cA < p.pitch && r0 < p.ny) {
        const unsigned o = (unsigned)r0 * (unsigned)p.pitch + (unsigned)cA;
        w.pinN = __ldg(p.pin_bits + (o >> 5));
    }
    return w;
}

// One warp's strip: columns [60 sx - 2, 60 sx + 62) walked down rows
// [r0 - 2, r0 + rows_per_warp) with a register window of rows r .. r+2 (row
// r+3 in flight).  Lane l holds the pair of columns (cA, cA + 1),
// cA = 60 sx - 2 + 2 l, and evaluates the six springs its two nodes own
// (Algorithm 1; the forward directions (0,+1), (0,+2), (+1,0), (+2,0),
// (+1,+1), (+1,-1)); the reaction of each spring reaches the other end
// through a shuffle (same row) or through the running sum of the reactions
// that the rows above send into the next row.  Rows r0 - 2 and r0 - 1 are the
// halo: they evaluate only the springs that end in row r0 or r0 + 1.  Then
// symplectic Euler with gravity, wind and pins (Section 3) writes rows
// [r0, r1) of the output state and, with a surface model, the nodes whose
// path box reaches the box of the mesh's vertices are appended to the collision list.
// The row loop is unrolled four times with the window's four row slots
// renamed at each step, so the window moves without register copies.
// DLR: output rows evaluate the (+1,-1) springs in the lane that receives
// them (see below); PMARK: the listing test on packed differences.  Each
// gives the same results either way and is chosen per kernel variant by
// measured time (they change the register allocation).
template <bool MESH, bool PER_SPRING, bool DLR = false, bool PMARK = false>
__device__ __forceinline__ void walk_strip(const StepParams &p, const float *__restrict__ in, float *__restrict__ out,
                                           float wbase, int sx, int sy, int lane, int cloth,
                                           float2 &fsum, const WalkStatics &ws)
{
    const long long st = p.stride;
    const unsigned st32 = (unsigned)st;
    const int cA = sx * STRIP_COLS - 2 + 2 * lane;  // column of node A (even)
    const int r0 = sy * p.rows_per_warp;
    const int r1 = min(r0 + p.rows_per_warp, p.ny);  // output rows [r0, r1)
    const bool colmem = cA >= 0 && cA < p.pitch;     // both columns addressable
    const int cmem = min(max(cA, 0), p.pitch - 2);   // the pair loaded (clamped)
    const bool out_lane = lane >= 1 && lane <= 30;
    auto colok = [&](int c) { return c >= 0 && c < p.nx; };
    const bool okA = out_lane && colok(cA), okB = out_lane && colok(cA + 1);

    // which of the lane's springs exist column-wise (both ends inside the
    // grid; A in the even bit, B in the odd bit of each pair): right, right2,
    // down (and down2), down-left; down-right exists where right does
    unsigned cm = 0u;
    if (!PER_SPRING) {
        cm = (colok(cA) && colok(cA + 1)) | (colok(cA + 1) && colok(cA + 2)) << 1 |
             (colok(cA) && colok(cA + 2)) << 2 | (colok(cA + 1) && colok(cA + 3)) << 3 |
             colok(cA) << 4 | colok(cA + 1) << 5 | (colok(cA) && colok(cA - 1)) << 6 |
             (colok(cA + 1) && colok(cA)) << 7;
    }
    // strips whose lanes all have every spring take the constants unmasked
    const bool edge_strip = !PER_SPRING && __any_sync(FULL, cm != 0xffu);
    auto cmask = [&](int b) {
        return make_float2((cm >> b) & 1u ? 1.0f : 0.0f, (cm >> (b + 1)) & 1u ? 1.0f : 0.0f);
    };

    // wind: sin(base + alpha_r + beta_c) from per-row and per-column tables of
    // (sin, cos) and the addition formula; depends only on (row, col, time)
    const float2 sinB = ws.sinB, cosB = ws.cosB;
    // per-row inputs, fetched one row ahead: the row's wind table entry and
    // the word holding its pin bits (shifted where it is used, so that no
    // instruction waits for the load until the next row)
    auto row_inputs = [&](int r, float2 &tr, unsigned &pinword) {
        tr = make_float2(0.0f, 1.0f);
        pinword = 0u;
        if (r < r1) {
            if (p.has_wind) tr = __ldg(p.wind_rows + r);
            if (p.pin_bits && colmem) {
                const unsigned o = (unsigned)r * (unsigned)p.pitch + (unsigned)cA;
                pinword = __ldg(p.pin_bits + (o >> 5));
            }
        }
    };
    // the time phase's sine and cosine: before the first loads in the DLR
    // walk, after them in the others (each the faster form there)
    float sinW = 0.0f, cosW = 1.0f;
    if (DLR && p.has_wind) sincosf(wbase, &sinW, &cosW);
    float2 trN = ws.trN;
    unsigned pinN = ws.pinN;

    int r = r0 - 2;
    // the window's four row slots and the two slots of lane+1's pair
    Node2 Pa = load_row(in, st32, r, p.ny, p.pitch, cmem);
    Node2 Pb = load_row(in, st32, r + 1, p.ny, p.pitch, cmem);
    Node2 Pc = load_row(in, st32, r + 2, p.ny, p.pitch, cmem);
    if (!DLR && p.has_wind) sincosf(wbase, &sinW, &cosW);
    Node2 Pd, Ne, Nf;
    // reactions sent into the next row by the rows above (springs (+1,0),
    // (+1,+1), (+1,-1) of row r-1 and (+2,0) of row r-2), and the (+2,0)
    // reactions of row r-1 (they reach row r+1)
    Vec2 A1 = {}, D2p = {};
    unsigned markA = 0u, markB = 0u;  // rows (r - r0 < 32) whose node needs the collision phase

    // PH 0: row r0-2 (only its (+2,0) spring reaches an output row);
    // PH 1: row r0-1 (its (+1,*) and (+2,0) springs); PH 2: output rows.
    // P0, P1, P2: rows r, r+1, r+2; P3 receives row r+3; N0: lane+1's pair of
    // row r (from the previous row); N1 receives lane+1's pair of row r+1.
    auto row = [&](auto phase, Node2 &P0, Node2 &P1, Node2 &P2, Node2 &P3, Node2 &N0, Node2 &N1) {
        constexpr int PH = decltype(phase)::value;
        P3 = load_row(in, st32, r + 3, p.ny, p.pitch, cmem);  // prefetch
        Node2 M1;  // lane-1's B, row r+1 (.y only; with DLR the halo row PH 1 only)
        if (PH >= 1) {
            N1.px = shfl_down2(P1.px, 1); N1.py = shfl_down2(P1.py, 1); N1.pz = shfl_down2(P1.pz, 1);
            N1.vx = shfl_down2(P1.vx, 1); N1.vy = shfl_down2(P1.vy, 1); N1.vz = shfl_down2(P1.vz, 1);
        }
        if (PH == 1 || (PH == 2 && !DLR)) {
            M1.px.y = __shfl_up_sync(FULL, P1.px.y, 1);
            M1.py.y = __shfl_up_sync(FULL, P1.py.y, 1);
            M1.pz.y = __shfl_up_sync(FULL, P1.pz.y, 1);
            M1.vx.y = __shfl_up_sync(FULL, P1.vx.y, 1);
            M1.vy.y = __shfl_up_sync(FULL, P1.vy.y, 1);
            M1.vz.y = __shfl_up_sync(FULL, P1.vz.y, 1);
        }

        float2 ksR, kdR, ksR2, kdR2, ksD, kdD, ksD2, kdD2, ksDR, kdDR, ksDL, kdDL;
        if (PER_SPRING) {
            // slot planes hold 0 for springs that do not exist
            ksR = kdR = ksD = kdD = ksDR = kdDR = ksDL = kdDL = ksR2 = kdR2 = ksD2 = kdD2 = bc(0.0f);
            if (r >= 0 && r < p.ny && colmem) {
                const unsigned o = (unsigned)r * (unsigned)p.pitch + (unsigned)cA;
                const float *ks = p.ks_slot, *kd = p.kd_slot;
                ksD2 = __ldg((const float2 *)(ks + (o + 5u * st32)));
                kdD2 = __ldg((const float2 *)(kd + (o + 5u * st32)));
                if (PH >= 1) {
                    ksD = __ldg((const float2 *)(ks + (o + st32)));
                    kdD = __ldg((const float2 *)(kd + (o + st32)));
                    ksDR = __ldg((const float2 *)(ks + (o + 2u * st32)));
                    kdDR = __ldg((const float2 *)(kd + (o + 2u * st32)));
                    ksDL = __ldg((const float2 *)(ks + (o + 3u * st32)));
                    kdDL = __ldg((const float2 *)(kd + (o + 3u * st32)));
                }
                if (PH == 2) {
                    ksR = __ldg((const float2 *)(ks + o));
                    kdR = __ldg((const float2 *)(kd + o));
                    ksR2 = __ldg((const float2 *)(ks + (o + 4u * st32)));
                    kdR2 = __ldg((const float2 *)(kd + (o + 4u * st32)));
                }
            }
        } else {
            ksR = ksD = bc(p.ks[0]);
            kdR = kdD = bc(p.kd[0]);
            ksDR = ksDL = bc(p.ks[1]);
            kdDR = kdDL = bc(p.kd[1]);
            ksR2 = ksD2 = bc(p.ks[2]);
            kdR2 = kdD2 = bc(p.kd[2]);
            if (edge_strip) {
                const float2 mR = cmask(0), mR2 = cmask(2), mD = cmask(4), mDL = cmask(6);
                ksR = mul2(ksR, mR); kdR = mul2(kdR, mR);
                ksDR = mul2(ksDR, mR); kdDR = mul2(kdDR, mR);
                ksR2 = mul2(ksR2, mR2); kdR2 = mul2(kdR2, mR2);
                ksD = mul2(ksD, mD); kdD = mul2(kdD, mD);
                ksD2 = mul2(ksD2, mD); kdD2 = mul2(kdD2, mD);
                ksDL = mul2(ksDL, mDL); kdDL = mul2(kdDL, mDL);
            }
            if (PH < 2) {
                // halo rows above the grid own no springs
                const float2 m0 = bc(r >= 0 ? 1.0f : 0.0f);
                ksD2 = mul2(ksD2, m0); kdD2 = mul2(kdD2, m0);
                ksD = mul2(ksD, m0); kdD = mul2(kdD, m0);
                ksDR = mul2(ksDR, m0); kdDR = mul2(kdDR, m0);
                ksDL = mul2(ksDL, m0); kdDL = mul2(kdDL, m0);
            }
            if (r + 2 >= p.ny) {
                // the grid's last two rows: no (+2,0) springs, and none of
                // (+1,*) from the last row
                const float2 m1 = bc(r + 1 < p.ny ? 1.0f : 0.0f);
                ksD2 = kdD2 = bc(0.0f);
                ksD = mul2(ksD, m1); kdD = mul2(kdD, m1);
                ksDR = mul2(ksDR, m1); kdDR = mul2(kdDR, m1);
                ksDL = mul2(ksDL, m1); kdDL = mul2(kdDL, m1);
            }
        }

        // the forward springs of the pair at row r; the node's own force is
        // summed in the order they complete, and each reaction leaves for its
        // receiving node as soon as it is known
        const Vec2 fD2 = spring2(P0, P2, ksD2, kdD2, p.L0[5]);  // (+2,0): reaches row r+2
        Vec2 own = fD2;
        Vec2 A1n = D2p;  // reactions for row r+1
        if (PH >= 1) {
            const Vec2 fD = spring2(P0, P1, ksD, kdD, p.L0[1]);  // (+1,0)
            own = vadd(own, fD);
            A1n = vadd(A1n, fD);
            const Vec2 fDR = spring2s(P0, P1, N1, ksDR, kdDR, p.L0[2]);  // (+1,+1): ends at (P1.y, N1.x)
            own = vadd(own, fDR);
            // down-right reactions for row r+1: A <- lane-1's B, B <- own A
            Vec2 nDR;
            nDR.x = make_float2(__shfl_up_sync(FULL, fDR.x.y, 1), fDR.x.x);
            nDR.y = make_float2(__shfl_up_sync(FULL, fDR.y.y, 1), fDR.y.x);
            nDR.z = make_float2(__shfl_up_sync(FULL, fDR.z.y, 1), fDR.z.x);
            A1n = vadd(A1n, nDR);
            if (PH == 1 || !DLR) {
                const Vec2 fDL = spring2s(P0, M1, P1, ksDL, kdDL, p.L0[3]);  // (+1,-1): ends at (M1.y, P1.x)
                own = vadd(own, fDL);
                // down-left reactions for row r+1: A <- own B, B <- lane+1's A
                Vec2 nDL;
                nDL.x = make_float2(fDL.x.y, __shfl_down_sync(FULL, fDL.x.x, 1));
                nDL.y = make_float2(fDL.y.y, __shfl_down_sync(FULL, fDL.y.x, 1));
                nDL.z = make_float2(fDL.z.y, __shfl_down_sync(FULL, fDL.z.x, 1));
                A1n = vadd(A1n, nDL);
            } else {
                // DLR output rows: the (+1,-1) springs of own B and of lane+1's A
                // (N0.x), both ending in this lane's row-r+1 pair, are
                // evaluated here from the same operands in the same order as
                // by their owners, so lane+1 receives its A's force instead of
                // this lane receiving lane-1's row-r+1 B; their constants are
                // those of the (+1,+1) springs of the pair (same type, same
                // column mask) or, per spring, the straddling pair of slots
                const float2 ksL = PER_SPRING ? make_float2(ksDL.y, __shfl_down_sync(FULL, ksDL.x, 1)) : ksDR;
                const float2 kdL = PER_SPRING ? make_float2(kdDL.y, __shfl_down_sync(FULL, kdDL.x, 1)) : kdDR;
                const Vec2 fL = spring2d(rdstr(P1.px, P0.px.y, N0.px.x), rdstr(P1.py, P0.py.y, N0.py.x),
                                         rdstr(P1.pz, P0.pz.y, N0.pz.x), rdstr(P1.vx, P0.vx.y, N0.vx.x),
                                         rdstr(P1.vy, P0.vy.y, N0.vy.x), rdstr(P1.vz, P0.vz.y, N0.vz.x), ksL, kdL,
                                         p.L0[3]);
                Vec2 fDL;  // per own node: A's from lane-1, B's from here
                fDL.x = make_float2(__shfl_up_sync(FULL, fL.x.y, 1), fL.x.x);
                fDL.y = make_float2(__shfl_up_sync(FULL, fL.y.y, 1), fL.y.x);
                fDL.z = make_float2(__shfl_up_sync(FULL, fL.z.y, 1), fL.z.x);
                own = vadd(own, fDL);
                A1n = vadd(A1n, fL);  // reactions for row r+1: A <- own B's, B <- lane+1's A's
            }
        }

        if (PH == 2) {
            const float2 tr = trN;
            const unsigned pinw = pinN >> (((unsigned)r * (unsigned)p.pitch + (unsigned)cA) & 31u);
            row_inputs(r + 1, trN, pinN);
            const Vec2 fR = spring2s(P0, P0, N0, ksR, kdR, p.L0[0]);  // (0,+1): ends at (P0.y, N0.x)
            own = vadd(own, fR);
            // reactions arriving at this row from the left neighbours' springs
            Vec2 back;  // right spring of (r, c-1): A <- lane-1's B, B <- own A
            back.x = make_float2(__shfl_up_sync(FULL, fR.x.y, 1), fR.x.x);
            back.y = make_float2(__shfl_up_sync(FULL, fR.y.y, 1), fR.y.x);
            back.z = make_float2(__shfl_up_sync(FULL, fR.z.y, 1), fR.z.x);
            const Vec2 fR2 = spring2(P0, N0, ksR2, kdR2, p.L0[4]);  // (0,+2)
            own = vadd(own, fR2);
            back = vadd(back, Vec2{shfl_up2(fR2.x, 1), shfl_up2(fR2.y, 1), shfl_up2(fR2.z, 1)});  // (r, c-2)

            // F = own forward springs - reactions of the springs that end here
            const Vec2 F = vsub(own, vadd(A1, back));

            float2 ax = fma2(F.x, bc(p.inv_mass), bc(p.g[0]));
            float2 ay = fma2(F.y, bc(p.inv_mass), bc(p.g[1]));
            float2 az = fma2(F.z, bc(p.inv_mass), bc(p.g[2]));
            if (p.has_wind) {
                // sin(a + b) = sin(a) cos(b) + cos(a) sin(b), a = base + alpha_r
                const float sinR = sinW * tr.y + cosW * tr.x;
                const float cosR = cosW * tr.y - sinW * tr.x;
                const float2 w = mul2(bc(p.w_amp), fma2(bc(cosR), sinB, mul2(bc(sinR), cosB)));
                ax = fma2(w, bc(p.w_dir[0]), ax);
                ay = fma2(w, bc(p.w_dir[1]), ay);
                az = fma2(w, bc(p.w_dir[2]), az);
            }
            const float2 dt = bc(p.dt);
            float2 wx = fma2(dt, ax, P0.vx), wy = fma2(dt, ay, P0.vy), wz = fma2(dt, az, P0.vz);
            float2 xx = fma2(dt, wx, P0.px), xy = fma2(dt, wy, P0.py), xz = fma2(dt, wz, P0.pz);
            if (pinw & 3u) {
                // pinned nodes move kinematically: x += dt u, v = u (u = 0: fixed)
                if (pinw & 1u) {
                    xx.x = fmaf(p.dt, p.pin_vel[0], P0.px.x); xy.x = fmaf(p.dt, p.pin_vel[1], P0.py.x);
                    xz.x = fmaf(p.dt, p.pin_vel[2], P0.pz.x);
                    wx.x = p.pin_vel[0]; wy.x = p.pin_vel[1]; wz.x = p.pin_vel[2];
                }
                if (pinw & 2u) {
                    xx.y = fmaf(p.dt, p.pin_vel[0], P0.px.y); xy.y = fmaf(p.dt, p.pin_vel[1], P0.py.y);
                    xz.y = fmaf(p.dt, p.pin_vel[2], P0.pz.y);
                    wx.y = p.pin_vel[0]; wy.y = p.pin_vel[1]; wz.y = p.pin_vel[2];
                }
            }
            if (MESH) {
                // nodes whose path box reaches the mesh's padded vertex box
                // are marked for the collision phase after the walk.  PMARK:
                // per axis, the path's box misses the mesh box when both ends
                // lie below its low face or both above its high face; for
                // finite values a rounded difference has the sign of the
                // exact one, so the signs of packed differences decide it
                bool needA, needB;
                if (PMARK) {
                    const uint2 ox = box_out_bits(P0.px, xx, p.mlo[0], p.mhi[0]);
                    const uint2 oy = box_out_bits(P0.py, xy, p.mlo[1], p.mhi[1]);
                    const uint2 oz = box_out_bits(P0.pz, xz, p.mlo[2], p.mhi[2]);
                    needA = okA && !(pinw & 1u) && !((ox.x | oy.x | oz.x) >> 31);
                    needB = okB && !(pinw & 2u) && !((ox.y | oy.y | oz.y) >> 31);
                } else {
                    needA = okA && !(pinw & 1u) && fmaxf(P0.px.x, xx.x) >= p.mlo[0] &&
                            fminf(P0.px.x, xx.x) <= p.mhi[0] && fmaxf(P0.py.x, xy.x) >= p.mlo[1] &&
                            fminf(P0.py.x, xy.x) <= p.mhi[1] && fmaxf(P0.pz.x, xz.x) >= p.mlo[2] &&
                            fminf(P0.pz.x, xz.x) <= p.mhi[2];
                    needB = okB && !(pinw & 2u) && fmaxf(P0.px.y, xx.y) >= p.mlo[0] &&
                            fminf(P0.px.y, xx.y) <= p.mhi[0] && fmaxf(P0.py.y, xy.y) >= p.mlo[1] &&
                            fminf(P0.py.y, xy.y) <= p.mhi[1] && fmaxf(P0.pz.y, xz.y) >= p.mlo[2] &&
                            fminf(P0.pz.y, xz.y) <= p.mhi[2];
                }
                markA |= (unsigned)needA << (r - r0);
                markB |= (unsigned)needB << (r - r0);
            }
            if (okA) {
                if (!okB) {  // B is padding: keep it zero
                    xx.y = xy.y = xz.y = wx.y = wy.y = wz.y = 0.0f;
                }
                fsum = add2(fsum, add2(add2(xx, xy), xz));
                const unsigned o = (unsigned)r * (unsigned)p.pitch + (unsigned)cA;
                if (p.vstar) {  // velocity after integration, before the response (adjoint recompute)
                    *(float2 *)(p.vstar + o) = wx;
                    *(float2 *)(p.vstar + (o + st32)) = wy;
                    *(float2 *)(p.vstar + (o + 2u * st32)) = wz;
                }
                *(float2 *)(out + o) = xx;
                *(float2 *)(out + (o + st32)) = xy;
                *(float2 *)(out + (o + 2u * st32)) = xz;
                *(float2 *)(out + (o + 3u * st32)) = wx;
                *(float2 *)(out + (o + 4u * st32)) = wy;
                *(float2 *)(out + (o + 5u * st32)) = wz;
            }
        }
        // reactions for the rows below
        if (PH >= 1) A1 = A1n;
        D2p = fD2;
        r++;
    };
    using PH0 = std::integral_constant<int, 0>;
    using PH1 = std::integral_constant<int, 1>;
    using PH2 = std::integral_constant<int, 2>;
    row(PH0(), Pa, Pb, Pc, Pd, Ne, Nf);
    row(PH1(), Pb, Pc, Pd, Pa, Nf, Ne);
    for (;;) {
        if (r >= r1) break;
        row(PH2(), Pc, Pd, Pa, Pb, Ne, Nf);
        if (r >= r1) break;
        row(PH2(), Pd, Pa, Pb, Pc, Nf, Ne);
        if (r >= r1) break;
        row(PH2(), Pa, Pb, Pc, Pd, Ne, Nf);
        if (r >= r1) break;
        row(PH2(), Pb, Pc, Pd, Pa, Nf, Ne);
    }

    if (MESH) {
        // append the marked nodes to the collision list, row by row so that
        // consecutive entries are neighbouring columns
        unsigned rows = __reduce_or_sync(FULL, markA | markB);
        const int cnt = __popc(markA) + __popc(markB);
        const int total = __reduce_add_sync(FULL, cnt);
        if (total > 0) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(p.coll_count, (unsigned)total);
            base = __shfl_sync(FULL, base, 0);
            while (rows) {
                const int b = __ffs((int)rows) - 1;
                rows &= rows - 1;
                const int a = (int)((markA >> b) & 1u), bb = (int)((markB >> b) & 1u);
                int inc = a + bb;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(FULL, inc, d);
                    if (lane >= d) inc += y;
                }
                const int row_total = __shfl_sync(FULL, inc, 31);
                unsigned w = base + (unsigned)(inc - a - bb);
                const int o = (r0 + b) * p.pitch + cA;
                if (a) {
                    p.coll_list[w] = o;
                    if (p.coll_cloth) p.coll_cloth[w] = cloth;
                    w++;
                }
                if (bb) {
                    p.coll_list[w] = o + 1;
                    if (p.coll_cloth) p.coll_cloth[w] = cloth;
                }
                base += (unsigned)row_total;
            }
        }
    }
}

// MESH: list the nodes near the surface model for the collision kernel,
// which then ends the substep.  EDGE (the edge narrow phase): list nothing
// (edge_list_kernel lists the nodes from the updated positions) and leave
// the substep to that phase's kernels.
template <bool MESH, bool PER_SPRING, bool EDGE = false>
__global__ void CLOTH_WALK_BOUNDS substep_kernel(const StepParams p)
{
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * WARPS_PER_CTA + (threadIdx.x >> 5);
    const bool active = warp < p.strips_x * p.strips_y;
    const int sx = active ? warp % p.strips_x : 0, sy = active ? warp / p.strips_x : 0;
    WalkStatics ws{};
    if (active) ws = walk_statics(p, sx, sy, lane);  // before the wait: static tables only
    pdl_wait();
    // Every lane reads the substep counter itself and, with the parity known
    // at launch (p.parity >= 0), picks its buffers without waiting for it:
    // the row loads then overlap the counter's read, which only the wind
    // phase and the end of the substep need.  The mesh walk (DLR) keeps the
    // counter read by one thread and the buffers picked from it: there the
    // other form spilled and was 1.6% slower.
    constexpr bool DLR = MESH && !EDGE && !PER_SPRING;
    unsigned long long k;
    float wbase;
    if (DLR) {
        __shared__ unsigned long long s_k;
        __shared__ float s_wbase;
        if (threadIdx.x == 0) {
            k = *(volatile unsigned long long *)&p.ctrl->k;
            s_k = k;
            s_wbase = p.has_wind ? wind_base(p.w_turn_step, p.w_turn0, k) : 0.0f;
        }
        __syncthreads();
        k = s_k;
        wbase = s_wbase;
    } else {
        k = *(volatile unsigned long long *)&p.ctrl->k;
        wbase = p.has_wind ? wind_base(p.w_turn_step, p.w_turn0, k) : 0.0f;
    }
    const bool odd = p.parity >= 0 && !DLR ? p.parity != 0 : (k & 1ull) != 0ull;
    const float *__restrict__ in = odd ? p.state1 : p.state0;
    float *__restrict__ out = odd ? p.state0 : p.state1;
    // sum of the stored positions: non-finite iff one of them is or a stored
    // velocity is (x = x0 + dt v with dt > 0; a pinned node's v is finite)
    float2 fsum = bc(0.0f);
    // DLR (receiver-side (+1,-1) springs) in the mesh walk only: 2% faster
    // there, slower without a mesh
    if (active) walk_strip<MESH && !EDGE, PER_SPRING, DLR>(p, in, out, wbase, sx, sy, lane, 0, fsum, ws);
    // the launch's parity checked against the counter after the walk (a
    // check before it would make the walk wait for the counter)
    if (!DLR && p.parity >= 0 && (int)(k & 1ull) != p.parity && threadIdx.x == 0)
        atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_PARITY);

    const bool bad = !isfinite(fsum.x + fsum.y);
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    if (MESH || EDGE) return;  // the collision kernels finish the substep
    __syncthreads();
    if (threadIdx.x == 0) {
        // the last CTA to finish advances the substep counter for the next launch
        const unsigned prev = atomicAdd(&p.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            p.ctrl->blocks_done = 0;
            p.ctrl->k = k + 1;
        }
    }
}

// Second kernel of a substep with a surface model: broad + narrow phase and
// response of every node the walk listed (warp-cooperative, collide_list),
// then the substep counter advances.

// List entries of one cloth.
struct OneClothList {
    const StepParams &p;
    __device__ void entry(unsigned long long i, int &cloth, long long &o) const
    {
        cloth = 0;
        o = __ldg(p.coll_list + i);
    }
    __device__ const StepParams &params(int) const { return p; }
};

// Collision pass over the nodes the walk listed (cooperative, see
// collide_list); the last CTA resets the list and advances the substep counter.
// REC: the adjoint recompute's variant, which also records each hit's
// response data (p.cdata, p.cbits).
template <bool REC>
__global__ void __launch_bounds__(32 * COLL_WARPS, CLOTH_COLL_MINB) collide_kernel(const __grid_constant__ StepParams p)
{
    __shared__ std::conditional_t<REC, CollSharedRec, CollShared> sh;
    __shared__ unsigned long long s_k;
    __shared__ unsigned s_n, s_stat[2];
    pdl_launch_dependents();
    pdl_wait();
    // the lane's first list entry, loaded beside the list length instead of
    // after it (the list holds p.n entries; one past the length is stale and
    // ignored)
    const unsigned long long i0 = coll_first_index();
    const long long pre_o = i0 < (unsigned long long)p.n ? (long long)__ldg(p.coll_list + i0) : 0ll;
    if (threadIdx.x == 0) {
        s_k = *(volatile unsigned long long *)&p.ctrl->k;
        s_n = *(volatile unsigned *)p.coll_count;
        s_stat[0] = s_stat[1] = 0u;
    }
    __syncthreads();
    const unsigned long long k = s_k;
    if (s_n == 0u) {
        // nothing listed (every CTA sees the same final count): CTA 0 alone
        // ends the substep; the others read k only to ignore it, and the
        // next kernel reads it after this grid completes
        if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->k = k + 1;
        return;
    }
    float fsum = 0.0f;
    unsigned ntest = 0u, nhit = 0u;
    collide_list<REC>(OneClothList{p}, sh, k, s_n, fsum, ntest, nhit, true, pre_o);
    if (__any_sync(FULL, !isfinite(fsum)) && (threadIdx.x & 31) == 0)
        atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    coll_stats_add(p.ctrl, s_stat, s_n, ntest, nhit);
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&p.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            p.ctrl->blocks_done = 0;
            *p.coll_count = 0u;
            p.ctrl->k = k + 1;
        }
    }
}

// Listing of the edge narrow phase: every node whose 3 x 3 block of
// nodes at the updated positions (the walk's output) has a box that reaches
// the (padded) box of the mesh's vertices.  A node is affected only through
// an edge of one of its triangles, all of whose vertices lie in that block,
// and such an edge can hit a triangle of the surface model only if its box
// meets the mesh's box; so every node a hit can affect is listed, however
// far the cloth is stretched.  Pinned nodes are listed too: their edges are
// tested (pass A) although they do not move.  Each listed node's stamp is set
// to the substep, which tells pass B whose edges were tested.  One thread per
// node; appends are aggregated per warp.
__global__ void __launch_bounds__(256) edge_list_kernel(const __grid_constant__ StepParams p)
{
    __shared__ unsigned long long s_k;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) s_k = *(volatile unsigned long long *)&p.ctrl->k;
    __syncthreads();
    const unsigned long long k = s_k;
    const float *xs = (k & 1ull) ? p.state0 : p.state1;  // updated positions
    const long long st = p.stride;
    const int lane = threadIdx.x & 31;
    const long long n = (long long)p.nx * p.ny;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < n; b += (long long)gridDim.x * blockDim.x) {
        const long long i = b + threadIdx.x;
        bool want = false;
        int o = 0;
        if (i < n) {
            const int r = (int)(i / p.nx), c = (int)(i - (long long)r * p.nx);
            o = r * p.pitch + c;
            {
                float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                for (int dr = -1; dr <= 1; dr++) {
                    const int rr = r + dr;
                    if (rr < 0 || rr >= p.ny) continue;
                    for (int dc = -1; dc <= 1; dc++) {
                        const int cc = c + dc;
                        if (cc < 0 || cc >= p.nx) continue;
                        const int q = rr * p.pitch + cc;
#pragma unroll
                        for (int a = 0; a < 3; a++) {
                            const float x = __ldg(xs + a * st + q);
                            lo[a] = fminf(lo[a], x);
                            hi[a] = fmaxf(hi[a], x);
                        }
                    }
                }
                want = lo[0] <= p.mhi[0] && hi[0] >= p.mlo[0] && lo[1] <= p.mhi[1] && hi[1] >= p.mlo[1] &&
                       lo[2] <= p.mhi[2] && hi[2] >= p.mlo[2];
            }
        }
        const unsigned m = __ballot_sync(FULL, want);
        if (m) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(p.coll_count, (unsigned)__popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (want) {
                p.coll_list[base + __popc(m & ((1u << lane) - 1u))] = o;
                p.edge_stamp[o] = k + 1ull;  // its owned edges get tested this substep
            }
        }
    }
}

// Edge narrow phase (CLOTH_FLAG_EDGE_COLLISION): pass A tests each listed
// node's owned edges and records their hits; pass B gathers every listed free
// node's response from the records of its 12 edges into a scratch array; a
// third kernel applies the responses, so no test reads a moved node.
__global__ void __launch_bounds__(32 * COLL_WARPS, CLOTH_COLL_MINB) edge_test_kernel(const __grid_constant__ StepParams p)
{
    __shared__ EdgeShared sh;
    __shared__ unsigned long long s_k;
    __shared__ unsigned s_n, s2[2];
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_k = *(volatile unsigned long long *)&p.ctrl->k;
        s_n = *(volatile unsigned *)p.coll_count;
        s2[0] = s2[1] = 0u;
    }
    __syncthreads();
    unsigned ntest = 0, nhit = 0;
    edge_test_list(p, sh, s_k, s_n, ntest, nhit);
    coll_stats_add(p.ctrl, s2, s_n, ntest, nhit);
}

__global__ void __launch_bounds__(256) edge_gather_kernel(const __grid_constant__ StepParams p)
{
    __shared__ unsigned long long s_k;
    __shared__ unsigned s_n;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_k = *(volatile unsigned long long *)&p.ctrl->k;
        s_n = *(volatile unsigned *)p.coll_count;
    }
    __syncthreads();
    edge_gather_list(p, s_k, s_n);
}

__global__ void __launch_bounds__(256) edge_apply_kernel(const __grid_constant__ StepParams p)
{
    __shared__ unsigned long long s_k;
    __shared__ unsigned s_n;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_k = *(volatile unsigned long long *)&p.ctrl->k;
        s_n = *(volatile unsigned *)p.coll_count;
    }
    __syncthreads();
    const unsigned long long k = s_k;
    float *out = (k & 1ull) ? p.state0 : p.state1;
    const long long st = p.stride;
    float fsum = 0.0f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < s_n; i += gridDim.x * blockDim.x) {
        const float4 e = p.edge_resp[i];
        if (e.w == 0.0f) continue;
        const int o = __ldg(p.coll_list + i);
        out[o] = e.x;
        out[st + o] = e.y;
        out[2 * st + o] = e.z;
        out[3 * st + o] *= p.restitution;
        out[4 * st + o] *= p.restitution;
        out[5 * st + o] *= p.restitution;
        fsum += e.x + e.y + e.z;
    }
    if (__any_sync(FULL, !isfinite(fsum)) && (threadIdx.x & 31) == 0)
        atomicOr(&p.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    __syncthreads();
    if (threadIdx.x == 0) {
        // the last CTA resets the list and advances the substep counter
        const unsigned prev = atomicAdd(&p.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            p.ctrl->blocks_done = 0;
            *p.coll_count = 0u;
            p.ctrl->k = k + 1;
        }
    }
}

// ---------------------------------------------------------------- batches
// Persistent walk over a list of (cloth, strip) items of many cloths: each
// warp takes the next item from a device counter (items sorted longest
// first), stages that cloth's parameters in its shared-memory slot and walks
// the strip with the same code as the single-cloth kernel, so every cloth of a
// batch gets exactly the arithmetic it gets when stepped alone.
// VAR: the walk variant every cloth of the batch shares (BATCH_VAR_MESH |
// BATCH_VAR_PER_SPRING), or BATCH_VAR_MIXED, which picks it per item; a
// kernel with one variant inlined holds fewer registers.
template <int VAR>
__global__ void __launch_bounds__(32 * CLOTH_WALK_WARPS, CLOTH_BATCH_MINB) batch_substep_kernel(const BatchArgs b)
{
    __shared__ StepParams sp[WARPS_PER_CTA];
    __shared__ unsigned long long s_k;
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) s_k = *(volatile unsigned long long *)&b.ctrl->k;
    __syncthreads();
    const unsigned long long k = s_k;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float2 fsum = bc(0.0f);
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(b.work, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= b.n_items) break;
        const int4 it = __ldg(b.items + item);  // (cloth, strip x, strip y, cost)
        const unsigned *src = (const unsigned *)(b.params + it.x);
        unsigned *dst = (unsigned *)&sp[wib];
        for (int w = lane; w < (int)(sizeof(StepParams) / 4); w += 32) dst[w] = __ldg(src + w);
        __syncwarp();
        const StepParams &p = sp[wib];
        const float wbase = p.has_wind ? wind_base(p.w_turn_step, p.w_turn0, k) : 0.0f;
        const float *in = (k & 1ull) ? p.state1 : p.state0;
        float *out = (k & 1ull) ? p.state0 : p.state1;
        const WalkStatics ws = walk_statics(p, it.y, it.z, lane);
        if (VAR != BATCH_VAR_MIXED) {
            // the packed listing test: 3.6% faster on config 5
            walk_strip<(VAR & BATCH_VAR_MESH) != 0, (VAR & BATCH_VAR_PER_SPRING) != 0, false, true>(
                p, in, out, wbase, it.y, it.z, lane, it.x, fsum, ws);
        } else if (p.has_mesh) {
            if (p.ks_slot) walk_strip<true, true>(p, in, out, wbase, it.y, it.z, lane, it.x, fsum, ws);
            else walk_strip<true, false>(p, in, out, wbase, it.y, it.z, lane, it.x, fsum, ws);
        } else {
            if (p.ks_slot) walk_strip<false, true>(p, in, out, wbase, it.y, it.z, lane, it.x, fsum, ws);
            else walk_strip<false, false>(p, in, out, wbase, it.y, it.z, lane, it.x, fsum, ws);
        }
        __syncwarp();  // the slot is rewritten by the next item
    }
    if (__any_sync(FULL, !isfinite(fsum.x + fsum.y)) && lane == 0)
        atomicOr(&b.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    __syncthreads();
    if (threadIdx.x == 0) {
        // the last CTA re-arms the work counter (the collision kernel advances k)
        const unsigned prev = atomicAdd(&b.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            b.ctrl->blocks_done = 0;
            *b.work = 0u;
        }
    }
}

// Collision kernel of a batch: every entry carries its cloth index.
// List entries of a batch: each carries its cloth.
struct BatchList {
    const BatchArgs &b;
    __device__ void entry(unsigned long long i, int &cloth, long long &o) const
    {
        cloth = __ldg(b.coll_cloth + i);
        o = __ldg(b.coll_list + i);
    }
    __device__ const StepParams &params(int c) const { return b.params[c]; }
};

__global__ void __launch_bounds__(32 * COLL_WARPS, CLOTH_COLL_MINB) batch_collide_kernel(const __grid_constant__ BatchArgs b)
{
    __shared__ CollShared sh;
    __shared__ unsigned long long s_k;
    __shared__ unsigned s_n, s_stat[2];
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_k = *(volatile unsigned long long *)&b.ctrl->k;
        s_n = *(volatile unsigned *)b.coll_count;
        s_stat[0] = s_stat[1] = 0u;
    }
    __syncthreads();
    const unsigned long long k = s_k;
    float fsum = 0.0f;
    unsigned ntest = 0u, nhit = 0u;
    collide_list(BatchList{b}, sh, k, s_n, fsum, ntest, nhit);
    if (__any_sync(FULL, !isfinite(fsum)) && (threadIdx.x & 31) == 0)
        atomicOr(&b.ctrl->flags, (unsigned)CTRL_FLAG_NONFINITE);
    coll_stats_add(b.ctrl, s_stat, s_n, ntest, nhit);
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&b.ctrl->blocks_done, 1u);
        if (prev == gridDim.x - 1) {
            b.ctrl->blocks_done = 0;
            *b.coll_count = 0u;
            b.ctrl->k = k + 1;
        }
    }
}

__global__ void aos_to_soa_kernel(const float *__restrict__ pos, const float *__restrict__ vel, float *state0,
                                  float *state1, long long st, int n, int nx, int pitch, DevCtrl *ctrl)
{
    const unsigned long long k = *(volatile unsigned long long *)&ctrl->k;
    float *dst = (k & 1ull) ? state1 : state0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long o = (long long)(i / nx) * pitch + (i % nx);
        if (pos) {
            dst[0 * st + o] = pos[3 * (long long)i];
            dst[1 * st + o] = pos[3 * (long long)i + 1];
            dst[2 * st + o] = pos[3 * (long long)i + 2];
        }
        if (vel) {
            dst[3 * st + o] = vel[3 * (long long)i];
            dst[4 * st + o] = vel[3 * (long long)i + 1];
            dst[5 * st + o] = vel[3 * (long long)i + 2];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->flags = 0u;
}

__global__ void soa_to_aos_kernel(const float *state0, const float *state1, long long st, int n, int nx, int pitch,
                                  const DevCtrl *ctrl, float *__restrict__ pos, float *__restrict__ vel)
{
    const unsigned long long k = *(volatile const unsigned long long *)&ctrl->k;
    const float *src = (k & 1ull) ? state1 : state0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long o = (long long)(i / nx) * pitch + (i % nx);
        if (pos) {
            pos[3 * (long long)i] = src[0 * st + o];
            pos[3 * (long long)i + 1] = src[1 * st + o];
            pos[3 * (long long)i + 2] = src[2 * st + o];
        }
        if (vel) {
            vel[3 * (long long)i] = src[3 * st + o];
            vel[3 * (long long)i + 1] = src[4 * st + o];
            vel[3 * (long long)i + 2] = src[5 * st + o];
        }
    }
}

int transfer_blocks(int n)
{
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

int substep_rows_per_warp(int nx, int ny, int sm_count)
{
    // the resident warps of one wave (register-limited), walks of 1..32 rows;
    // a walk of R rows takes R + 2 row iterations, so a grid that does not
    // fill a wave takes the shortest walks (128 x 128 with an icosphere, µs
    // per substep: R = 4 12.4, R = 2 10.0, R = 1 8.8)
    const long long strips_x = (nx + STRIP_COLS - 1) / STRIP_COLS;
    const long long target = (long long)sm_count * WARPS_PER_CTA * substep_min_ctas();
    long long strips_y = (target + strips_x - 1) / strips_x;
    long long R = (ny + strips_y - 1) / strips_y;
    if (R < 1) R = 1;
    if (R > CLOTH_MAX_ROWS_PER_WARP) R = CLOTH_MAX_ROWS_PER_WARP;
    return (int)R;
}

void substep_shape(StepParams &p)
{
    p.strips_x = (p.nx + STRIP_COLS - 1) / STRIP_COLS;
    p.strips_y = (p.ny + p.rows_per_warp - 1) / p.rows_per_warp;
}

namespace {
// Kernel launch with the programmatic-serialisation attribute (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), int blocks, int threads, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = CLOTH_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
}  // namespace

cudaError_t launch_walk(const StepParams &p, cudaStream_t s)
{
    if (p.force) return launch_atomic_forces_and_integrate(p, s);
    const int warps = p.strips_x * p.strips_y;
    const int blocks = (warps + WARPS_PER_CTA - 1) / WARPS_PER_CTA;
    const bool per = p.ks_slot != nullptr;
    const int threads = 32 * WARPS_PER_CTA;
    if (p.has_mesh && p.edge_resp)
        return per ? launch_k(substep_kernel<true, true, true>, blocks, threads, s, p)
                   : launch_k(substep_kernel<true, false, true>, blocks, threads, s, p);
    if (p.has_mesh)
        return per ? launch_k(substep_kernel<true, true>, blocks, threads, s, p)
                   : launch_k(substep_kernel<true, false>, blocks, threads, s, p);
    return per ? launch_k(substep_kernel<false, true>, blocks, threads, s, p)
               : launch_k(substep_kernel<false, false>, blocks, threads, s, p);
}


cudaError_t launch_collide(const StepParams &p, cudaStream_t s)
{
    if (p.edge_resp) {
        cudaError_t e = launch_k(edge_list_kernel, p.coll_blocks, 256, s, p);
        if (e != cudaSuccess) return e;
        e = launch_k(edge_test_kernel, p.coll_blocks, 32 * COLL_WARPS, s, p);
        if (e != cudaSuccess) return e;
        e = launch_k(edge_gather_kernel, p.coll_blocks, 256, s, p);
        if (e != cudaSuccess) return e;
        return launch_k(edge_apply_kernel, p.coll_blocks, 256, s, p);
    }
    if (p.cdata) return launch_k(collide_kernel<true>, p.coll_blocks, 32 * COLL_WARPS, s, p);
    return launch_k(collide_kernel<false>, p.coll_blocks, 32 * COLL_WARPS, s, p);
}

cudaError_t launch_substep(const StepParams &p, cudaStream_t s)
{
    cudaError_t e = launch_walk(p, s);
    if (e == cudaSuccess && p.has_mesh) e = launch_collide(p, s);
    return e;
}

cudaError_t launch_batch_substep(const BatchArgs &b, cudaStream_t s)
{
    cudaError_t e;
    switch (b.variant) {
    case 0: e = launch_k(batch_substep_kernel<0>, b.walk_blocks, 32 * WARPS_PER_CTA, s, b); break;
    case BATCH_VAR_MESH: e = launch_k(batch_substep_kernel<BATCH_VAR_MESH>, b.walk_blocks, 32 * WARPS_PER_CTA, s, b); break;
    case BATCH_VAR_PER_SPRING:
        e = launch_k(batch_substep_kernel<BATCH_VAR_PER_SPRING>, b.walk_blocks, 32 * WARPS_PER_CTA, s, b);
        break;
    case BATCH_VAR_MESH | BATCH_VAR_PER_SPRING:
        e = launch_k(batch_substep_kernel<BATCH_VAR_MESH | BATCH_VAR_PER_SPRING>, b.walk_blocks, 32 * WARPS_PER_CTA,
                     s, b);
        break;
    default: e = launch_k(batch_substep_kernel<BATCH_VAR_MIXED>, b.walk_blocks, 32 * WARPS_PER_CTA, s, b); break;
    }
    if (e != cudaSuccess) return e;
    return launch_k(batch_collide_kernel, b.coll_blocks, 32 * COLL_WARPS, s, b);
}

int substep_strip_cols() { return STRIP_COLS; }
int substep_warps_per_cta() { return WARPS_PER_CTA; }
// Resident CTAs per SM of the single-cloth walk kernel and of the batch walk
// kernel, from the occupancy calculator; looked up once each.
namespace {
int occupancy(const void *kern, int fallback)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * WARPS_PER_CTA, 0) != cudaSuccess) {
        cudaGetLastError();
        return fallback;
    }
    return n < 1 ? 1 : n;
}
}  // namespace

int substep_min_ctas()
{
    static int cached = 0;
    if (cached <= 0) cached = occupancy((const void *)substep_kernel<true, false>, CLOTH_WALK_MINB);
    return cached;
}

int batch_min_ctas()
{
    static int cached = 0;
    // the most register-hungry of the variants (they share the launch bounds)
    if (cached <= 0) cached = occupancy((const void *)batch_substep_kernel<BATCH_VAR_MIXED>, CLOTH_BATCH_MINB);
    return cached;
}

cudaError_t launch_aos_to_soa(const float *aos_pos, const float *aos_vel, float *state0, float *state1,
                              long long stride, int n, int nx, int pitch, DevCtrl *ctrl, cudaStream_t s)
{
    aos_to_soa_kernel<<<transfer_blocks(n), 256, 0, s>>>(aos_pos, aos_vel, state0, state1, stride, n, nx, pitch,
                                                         ctrl);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const float *state0, const float *state1, long long stride, int n, int nx, int pitch,
                              const DevCtrl *ctrl, float *aos_pos, float *aos_vel, cudaStream_t s)
{
    soa_to_aos_kernel<<<transfer_blocks(n), 256, 0, s>>>(state0, state1, stride, n, nx, pitch, ctrl, aos_pos,
                                                         aos_vel);
    return cudaGetLastError();
}
