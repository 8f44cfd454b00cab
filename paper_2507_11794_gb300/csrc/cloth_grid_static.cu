// cloth_grid_build_static: the uniform-grid build of cloth_set_mesh for
// callers that cannot allocate device memory -- hosts that run under an
// allocator with a fixed budget, or that forbid cudaMalloc/cudaFree once
// start-up is over.  All temporaries live in one file-scope device array of
// fixed size, so this entry point allocates nothing; the caller supplies the
// output buffers.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "cloth_internal.h"

namespace {

constexpr long long kMaxTris = CLOTH_STATIC_GRID_MAX_TRIS;
constexpr long long kMaxVerts = CLOTH_STATIC_GRID_MAX_VERTS;
constexpr long long kMaxCells = CLOTH_STATIC_GRID_MAX_CELLS;
constexpr long long kTiles = (kMaxCells + 1023) / 1024;

// Byte offsets of the temporaries inside the scratch array (256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffVerts = 0;
constexpr size_t kOffTris = align256(kOffVerts + sizeof(float) * 3 * kMaxVerts);
constexpr size_t kOffBoxHi = align256(kOffTris + sizeof(int) * 3 * kMaxTris);
constexpr size_t kOffCnt = align256(kOffBoxHi + sizeof(int4) * kMaxTris);
constexpr size_t kOffCursor = align256(kOffCnt + sizeof(unsigned) * kMaxCells);
constexpr size_t kOffSums = align256(kOffCursor + sizeof(unsigned) * kMaxCells);
constexpr size_t kOffTotal = align256(kOffSums + sizeof(unsigned) * kTiles);
constexpr size_t kScratchBytes = align256(kOffTotal + sizeof(unsigned long long));

// A device holds this array from the moment the library's module is loaded on
// it (with CUDA's lazy module loading, at the first use of the library on that
// device, which may be the first call below) until the process exits.
static __device__ __align__(256) unsigned char g_grid_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

int fail(int code, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    cloth_set_error_message(msg);
    return code;
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
cudaError_t scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = (unsigned char *)g_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int cloth_grid_build_static(const float *verts, int32_t nverts, const int32_t *tris, int32_t ntris,
                                       void *stream, float *d_tri_records, int32_t *d_cell_start,
                                       int64_t cell_capacity, int32_t *d_tri_ids, int64_t entry_capacity,
                                       ClothGridParams *params)
{
    if (!params) return fail(CLOTH_ERR_INVALID_ARG, "params is NULL");
    params->nentries = -1;
    params->ncells = 0;
    if (!verts || !tris || ntris < 1 || nverts < 1) return fail(CLOTH_ERR_INVALID_ARG, "empty or missing mesh");
    if (ntris > kMaxTris || nverts > kMaxVerts)
        return fail(CLOTH_ERR_INVALID_ARG, "mesh of %d triangles / %d vertices exceeds the static limits (%lld / %lld)",
                    ntris, nverts, kMaxTris, kMaxVerts);
    for (long long i = 0; i < 3 * (long long)ntris; i++)
        if (tris[i] < 0 || tris[i] >= nverts)
            return fail(CLOTH_ERR_BAD_MESH, "triangle index %d at %lld out of range [0, %d)", tris[i], i, nverts);
    for (long long i = 0; i < 3 * (long long)nverts; i++)
        if (!isfinite(verts[i])) return fail(CLOTH_ERR_BAD_MESH, "non-finite vertex coordinate at %lld", i);
    int dims[3];
    if (grid_params(verts, tris, ntris, &params->h, params->origin, dims, &params->inv) != 0)
        return fail(CLOTH_ERR_BAD_MESH, "grid parameters");
    for (int a = 0; a < 3; a++) params->dims[a] = dims[a];
    params->ncells = (int64_t)dims[0] * dims[1] * dims[2];
    if (params->ncells > kMaxCells)
        return fail(CLOTH_ERR_INVALID_ARG, "grid of %lld cells exceeds the static limit (%lld)",
                    (long long)params->ncells, kMaxCells);
    if (!d_tri_records || ((uintptr_t)d_tri_records & 15u))
        return fail(CLOTH_ERR_INVALID_ARG, "d_tri_records must be a 16-byte aligned device buffer of 12*ntris floats");
    if (!d_cell_start || cell_capacity < params->ncells + 1)
        return fail(CLOTH_ERR_INVALID_ARG, "d_cell_start holds %lld ints, needs %lld", (long long)cell_capacity,
                    (long long)params->ncells + 1);
    if (entry_capacity > 0 && !d_tri_ids) return fail(CLOTH_ERR_INVALID_ARG, "d_tri_ids is NULL");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CLOTH_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(CLOTH_ERR_INVALID_ARG, "device %d: the static grid build serves devices 0..%d", dev,
                    kMaxDevices - 1);
    unsigned char *base = nullptr;
    if ((e = scratch_address(dev, &base)) != cudaSuccess)
        return fail(CLOTH_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    float *sv = (float *)(base + kOffVerts);
    int *st = (int *)(base + kOffTris);
    if ((e = cudaMemcpyAsync(sv, verts, sizeof(float) * 3 * (size_t)nverts, cudaMemcpyHostToDevice, s)) ==
            cudaSuccess &&
        (e = cudaMemcpyAsync(st, tris, sizeof(int) * 3 * (size_t)ntris, cudaMemcpyHostToDevice, s)) == cudaSuccess) {
        long long nent = 0;
        bool done = false;
        e = grid_build_noalloc(sv, st, ntris, params->origin, params->inv, dims, (float4 *)d_tri_records,
                               d_cell_start, d_tri_ids, entry_capacity, (int4 *)(base + kOffBoxHi),
                               (unsigned *)(base + kOffCnt), (unsigned *)(base + kOffCursor),
                               (unsigned *)(base + kOffSums), (unsigned long long *)(base + kOffTotal), &nent, &done,
                               s);
        if (e == cudaSuccess) {
            params->nentries = nent;
            if (nent >= 0x7fffffffLL)  // cell_start and tri_ids are int32
                return fail(CLOTH_ERR_BAD_MESH, "%lld (cell, triangle) pairs: more than int32 indices address",
                            nent);
            if (!done)
                return fail(CLOTH_ERR_INVALID_ARG, "d_tri_ids holds %lld ints, needs %lld",
                            (long long)entry_capacity, nent);
            return CLOTH_OK;
        }
    }
    return fail(CLOTH_ERR_CUDA, "static grid build: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
}
