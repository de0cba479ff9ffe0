// C ABI of the single-channel solver (declared in include/lbm.h): handle
// management, step orchestration with CUDA graphs, statistics and exports.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "lbm.h"
#include "lbm_quad.cuh"
#include "lbm_tma.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CK_LAUNCH() CK(cudaGetLastError())

constexpr int kGraphSteps = 16;   // steps captured per chunk graph (even)

}  // namespace

#include "lbm_handle.h"

int lbm_record_error(int code, const char *msg) { return fail(code, "%s", msg); }

namespace {

size_t elem_size(const lbm_handle *h) { return h->precision == LBM_FP16_SHIFTED ? 2 : 4; }

dim3 grid_of(const lbm_handle *h, int bx) { return dim3((h->g.nx + bx - 1) / bx, h->g.ny, h->g.nz); }

// grid of the step kernel: one thread per cell, or per x-pair for even nx
int cells_per_thread(int kernel) { return kernel == LBM_KERNEL_CELL ? 1 : (kernel == LBM_KERNEL_QUAD ? 4 : 2); }

dim3 step_grid(const lbm_handle *h)
{
    const int per_row = h->g.nx / cells_per_thread(h->kernel);
    return dim3((per_row + h->bx - 1) / h->bx, h->g.ny, h->g.nz);
}

int configure_rows(lbm_handle *h);

int select_kernel(lbm_handle *h, int kernel)
{
    const bool even = (h->g.nx % 2) == 0;
    const bool seg = (h->g.nx % 64) == 0;
    // wall nodes: every form but the row pipeline (the four-cell step runs its
    // node rows with the two-cell wall tile)
    const bool node = h->p.wall == lbm::WALL_NODE;
    const bool quad = (h->g.nx % 4) == 0 && h->precision == LBM_FP16_SHIFTED;
    // AUTO: FP16 storage with nx a multiple of 4 runs the four-cell kernel, else
    // the two-cell kernel where nx is even, else the one-cell kernel (measured
    // fastest in that order on GB300 for every benchmark grid)
    if (kernel == LBM_KERNEL_AUTO) kernel = quad ? LBM_KERNEL_QUAD : (even ? LBM_KERNEL_PAIR : LBM_KERNEL_CELL);
    if (kernel == LBM_KERNEL_PAIR && !even) return fail(LBM_ERR_ARG, "two-cell kernel needs an even nx");
    if (kernel == LBM_KERNEL_QUAD && !quad)
        return fail(LBM_ERR_ARG, "four-cell kernel needs FP16 storage and nx a multiple of 4");
    if (kernel == LBM_KERNEL_TMA && node) return fail(LBM_ERR_ARG, "the pipelined kernel has no wall-node form");
    if (kernel == LBM_KERNEL_TMA && !seg) return fail(LBM_ERR_ARG, "pipelined kernel needs nx a multiple of 64");
    if (kernel == LBM_KERNEL_TMA && h->layout == LBM_AA)
        return fail(LBM_ERR_ARG, "the AA layout runs the cell, pair or quad kernel");
    if (kernel < LBM_KERNEL_CELL || kernel > LBM_KERNEL_QUAD) return fail(LBM_ERR_ARG, "unknown kernel");
    h->kernel = kernel;
    const int per_row = h->g.nx / cells_per_thread(kernel);
    h->bx = per_row >= 128 ? 128 : (per_row > 32 ? 64 : 32);   // <= the kernels' launch bound of 128
    if (kernel == LBM_KERNEL_TMA) {
        const int rc = configure_rows(h);
        if (rc != LBM_OK) return rc;
    }
    // captured graphs hold the old launch configuration
    for (int i = 0; i < 2; ++i)
        if (h->chunk[i]) {
            cudaGraphExecDestroy(h->chunk[i]);
            h->chunk[i] = nullptr;
        }
    return LBM_OK;
}

// Read (and clear) the device flag of a timed-out pipeline wait: a timeout is
// reported once, by the first synchronising call after it.
int check_err(lbm_handle *h)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e) {
        CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return fail(LBM_ERR_CUDA, "a pipeline wait in the step kernel timed out");
    }
    return LBM_OK;
}

// block partials of one sampled step, per wall-normal plane
long long partials_per_plane(const lbm_handle *h)
{
    if (h->kernel == LBM_KERNEL_TMA) return (long long)h->tma_warps * h->g.nz;
    return (long long)step_grid(h).x * h->g.nz;
}

#ifndef LBM_FORK_WALL
#define LBM_FORK_WALL 1
#endif

// Launch with programmatic stream serialisation (see pdl_begin in
// lbm_pair.cuh) when pdl is set: the grid starts while the previous kernel on
// the stream drains. Kernels that read the previous step's output through the
// read-only path launch without it (pull_nc in lbm_device.cuh).
template <typename... K, typename... A>
cudaError_t launch_ex(bool pdl, void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args)
{
    return launch_ex(true, kernel, grid, block, smem, s, args...);
}

template <typename T, int NW, int COLL>
void launch_rows_t(lbm_handle *h, cudaStream_t s, int src, bool stats)
{
    const T *a = (const T *)h->f[src];
    T *b = (T *)h->f[src ^ 1];
    const dim3 grid(h->tma_grid), block(NW * 32);
    if (stats)
        lbm::k_step_rows<T, true, NW, COLL><<<grid, block, h->tma_smem, s>>>(a, b, h->g, h->p, h->tw, h->part, h->err,
                                                                              h->tma_stages, h->wait_limit);
    else
        lbm::k_step_rows<T, false, NW, COLL><<<grid, block, h->tma_smem, s>>>(a, b, h->g, h->p, h->tw, h->part,
                                                                               h->err, h->tma_stages, h->wait_limit);
}

// Blocks per SM of one row-kernel instantiation with `smem` dynamic bytes.
template <typename T, int NW, int COLL>
int rows_occupancy_c(int smem, int *per_sm)
{
    CK(cudaFuncSetAttribute(lbm::k_step_rows<T, false, NW, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(lbm::k_step_rows<T, true, NW, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, lbm::k_step_rows<T, false, NW, COLL>, NW * 32, smem));
    int st = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&st, lbm::k_step_rows<T, true, NW, COLL>, NW * 32, smem));
    *per_sm = std::min(*per_sm, st);
    return LBM_OK;
}

int rows_occupancy(const lbm_handle *h, int nw, int smem, int *per_sm)
{
    const bool half = h->precision == LBM_FP16_SHIFTED, mrt = h->p.collision == lbm::COLL_MRT;
    if (half) {
        if (mrt)
            return nw == 8 ? rows_occupancy_c<__half, 8, lbm::COLL_MRT>(smem, per_sm)
                           : rows_occupancy_c<__half, 4, lbm::COLL_MRT>(smem, per_sm);
        return nw == 8 ? rows_occupancy_c<__half, 8, lbm::COLL_BGK>(smem, per_sm)
                       : rows_occupancy_c<__half, 4, lbm::COLL_BGK>(smem, per_sm);
    }
    if (mrt)
        return nw == 8 ? rows_occupancy_c<float, 8, lbm::COLL_MRT>(smem, per_sm)
                       : rows_occupancy_c<float, 4, lbm::COLL_MRT>(smem, per_sm);
    return nw == 8 ? rows_occupancy_c<float, 8, lbm::COLL_BGK>(smem, per_sm)
                   : rows_occupancy_c<float, 4, lbm::COLL_BGK>(smem, per_sm);
}

// Warps per CTA, ring depth and grid of the row kernel: the most resident
// warps per SM, then the deepest ring. Fails if even two stages do not fit.
int configure_rows(lbm_handle *h)
{
    int dev = 0, sms = 0, smem_max = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const bool half = h->precision == LBM_FP16_SHIFTED;
    const int nw = h->g.nx >= 512 ? 8 : 4;
    int best_warps = 0, best_stages = 0, best_per_sm = 0;
    for (int stages = lbm::ROW_MAX_STAGES; stages >= 2; --stages) {
        const int smem = half ? lbm::rows_smem_bytes<__half>(h->g.nx, stages)
                              : lbm::rows_smem_bytes<float>(h->g.nx, stages);
        if (smem > smem_max) continue;
        int per_sm = 0;
        const int rc = rows_occupancy(h, nw, smem, &per_sm);
        if (rc != LBM_OK) return rc;
        if (per_sm * nw > best_warps) {
            best_warps = per_sm * nw;
            best_stages = stages;
            best_per_sm = per_sm;
        }
    }
    if (best_warps == 0) return fail(LBM_ERR_ARG, "rows of this grid do not fit the pipelined kernel's shared memory");
    h->tma_warps = nw;
    h->tma_stages = best_stages;
    h->tma_smem = half ? lbm::rows_smem_bytes<__half>(h->g.nx, best_stages)
                       : lbm::rows_smem_bytes<float>(h->g.nx, best_stages);
    h->tma_grid = sms * best_per_sm;
    // the probe above left the attribute at the last candidate: set the chosen size
    int per_sm = 0;
    return rows_occupancy(h, nw, h->tma_smem, &per_sm);
}

// One step with the kernel form of the handle, collision operator COLL.
// One in-place AA step of kind LAY (even from phase 0, odd from phase 1).
template <int COLL, int LAY>
cudaError_t launch_aa(lbm_handle *h, cudaStream_t s, bool stats)
{
    const dim3 grid = step_grid(h), block(h->bx);
    void *f = h->f[0];
    if (h->kernel == LBM_KERNEL_QUAD) {
        __half *fh = (__half *)f;
        // The odd step (gather and push through the neighbours, the heavier
        // kind) calls a separately compiled wall-row tile, which frees the
        // interior's registers (c4 FP16: 1.96 against 2.11 ms); the even step
        // is measured faster with the wall layer inline (1.62 against 1.67 ms).
        // Both are one launch over every row: an interior / wall-row split,
        // as in the two-lattice step, measured slower in place.
        if constexpr (LAY == lbm::LAY_AA_ODD)
            if (!stats && h->g.ny > 2)
                return launch_pdl(lbm::k_step_quad_aa_rows<false, COLL, LAY>, grid, block, 0, s, fh, h->g, h->p,
                                  h->tw, h->part);
        return stats ? launch_pdl(lbm::k_step_quad_aa<true, COLL, LAY>, grid, block, 0, s, fh, h->g, h->p, h->tw, h->part)
                     : launch_pdl(lbm::k_step_quad_aa<false, COLL, LAY>, grid, block, 0, s, fh, h->g, h->p, h->tw,
                                  h->part);
    }
    if (h->kernel == LBM_KERNEL_PAIR) {
        if (h->precision == LBM_FP16_SHIFTED) {
            __half *fh = (__half *)f;
            return stats ? launch_pdl(lbm::k_step_pair_aa<__half, true, COLL, LAY>, grid, block, 0, s, fh, h->g, h->p,
                                      h->tw, h->part)
                         : launch_pdl(lbm::k_step_pair_aa<__half, false, COLL, LAY>, grid, block, 0, s, fh, h->g, h->p,
                                      h->tw, h->part);
        }
        float *ff = (float *)f;
        return stats ? launch_pdl(lbm::k_step_pair_aa<float, true, COLL, LAY>, grid, block, 0, s, ff, h->g, h->p, h->tw,
                                  h->part)
                     : launch_pdl(lbm::k_step_pair_aa<float, false, COLL, LAY>, grid, block, 0, s, ff, h->g, h->p,
                                  h->tw, h->part);
    }
    if (h->precision == LBM_FP16_SHIFTED) {
        if (stats)
            lbm::k_step_aa<__half, true, COLL, LAY><<<grid, block, 0, s>>>((__half *)f, h->g, h->p, h->tw, h->part);
        else
            lbm::k_step_aa<__half, false, COLL, LAY><<<grid, block, 0, s>>>((__half *)f, h->g, h->p, h->tw, h->part);
    } else {
        if (stats)
            lbm::k_step_aa<float, true, COLL, LAY><<<grid, block, 0, s>>>((float *)f, h->g, h->p, h->tw, h->part);
        else
            lbm::k_step_aa<float, false, COLL, LAY><<<grid, block, 0, s>>>((float *)f, h->g, h->p, h->tw, h->part);
    }
    return cudaSuccess;
}

template <int COLL>
int launch_step_c(lbm_handle *h, cudaStream_t s, int src, bool stats, cudaStream_t s_wall)
{
    const dim3 grid = step_grid(h), block(h->bx);
    const bool half = h->precision == LBM_FP16_SHIFTED;
    const void *a = h->f[src];
    void *b = h->f[src ^ 1];
    cudaError_t e = cudaSuccess;
    if (h->layout == LBM_AA) {
        // src is the phase: 0 runs the even step, 1 the odd step
        e = src == 0 ? launch_aa<COLL, lbm::LAY_AA_EVEN>(h, s, stats) : launch_aa<COLL, lbm::LAY_AA_ODD>(h, s, stats);
    } else if (h->kernel == LBM_KERNEL_TMA) {
        if (half) {
            if (h->tma_warps == 8)
                launch_rows_t<__half, 8, COLL>(h, s, src, stats);
            else
                launch_rows_t<__half, 4, COLL>(h, s, src, stats);
        } else {
            if (h->tma_warps == 8)
                launch_rows_t<float, 8, COLL>(h, s, src, stats);
            else
                launch_rows_t<float, 4, COLL>(h, s, src, stats);
        }
    } else if (h->kernel == LBM_KERNEL_QUAD) {
        // BGK: the interior rows, then the two wall rows with the two-cell tile
        // in CTAs of twice the threads (the wall layer lives only in the second
        // launch); MRT: one launch whose wall-row CTAs call a separately
        // compiled wall tile (k_step_quad_rows), measured 1-2% faster for MRT
        // and 8% slower for BGK than the two launches
        const __half *ah = (const __half *)a;
        __half *bh = (__half *)b;
        bool fused = false;
        if constexpr (COLL == lbm::COLL_MRT) {
            fused = h->g.ny > 2 && h->p.wall != lbm::WALL_NODE;   // the called wall tile has no node form
            if (fused)
                e = stats ? launch_pdl(lbm::k_step_quad_rows<true, COLL>, grid, block, 0, s, ah, bh, h->g, h->p,
                                       h->tw, h->part)
                          : launch_pdl(lbm::k_step_quad_rows<false, COLL>, grid, block, 0, s, ah, bh, h->g, h->p,
                                       h->tw, h->part);
        }
        if (!fused) {
            // the interior rows (BGK, or MRT with wall nodes), then the wall rows
            if (h->g.ny > 2) {
                const dim3 gi(grid.x, h->g.ny - 2, grid.z);
                e = stats ? launch_pdl(lbm::k_step_quad<true, COLL, lbm::ROWS_INTERIOR>, gi, block, 0, s, ah, bh,
                                       h->g, h->p, h->tw, h->part)
                          : launch_pdl(lbm::k_step_quad<false, COLL, lbm::ROWS_INTERIOR>, gi, block, 0, s, ah, bh,
                                       h->g, h->p, h->tw, h->part);
            }
            const dim3 gw(grid.x, 2, grid.z), bw(2 * h->bx);
            if (e == cudaSuccess)
                e = stats ? launch_pdl(lbm::k_step_pair_wall<__half, true, COLL>, gw, bw, 0, s_wall, ah, bh, h->g,
                                       h->p, h->tw, h->part)
                          : launch_pdl(lbm::k_step_pair_wall<__half, false, COLL>, gw, bw, 0, s_wall, ah, bh, h->g,
                                       h->p, h->tw, h->part);
        }
    } else if (h->kernel == LBM_KERNEL_PAIR) {
        if (half) {
            const __half *ah = (const __half *)a;
            __half *bh = (__half *)b;
            e = stats ? launch_pdl(lbm::k_step_pair<__half, true, COLL>, grid, block, 0, s, ah, bh, h->g, h->p, h->tw,
                                   h->part)
                      : launch_pdl(lbm::k_step_pair<__half, false, COLL>, grid, block, 0, s, ah, bh, h->g, h->p, h->tw,
                                   h->part);
        } else {
            const float *af = (const float *)a;
            float *bf = (float *)b;
            // read-only loads of the source lattice: no programmatic dependent launch
            e = stats ? launch_ex(false, lbm::k_step_pair<float, true, COLL>, grid, block, 0, s, af, bf, h->g, h->p, h->tw,
                                   h->part)
                      : launch_ex(false, lbm::k_step_pair<float, false, COLL>, grid, block, 0, s, af, bf, h->g, h->p, h->tw,
                                   h->part);
        }
    } else if (half) {
        if (stats)
            lbm::k_step<__half, true, COLL><<<grid, block, 0, s>>>((const __half *)a, (__half *)b, h->g, h->p, h->tw,
                                                                   h->part);
        else
            lbm::k_step<__half, false, COLL><<<grid, block, 0, s>>>((const __half *)a, (__half *)b, h->g, h->p, h->tw,
                                                                    h->part);
    } else {
        if (stats)
            lbm::k_step<float, true, COLL><<<grid, block, 0, s>>>((const float *)a, (float *)b, h->g, h->p, h->tw,
                                                                  h->part);
        else
            lbm::k_step<float, false, COLL><<<grid, block, 0, s>>>((const float *)a, (float *)b, h->g, h->p, h->tw,
                                                                   h->part);
    }
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "step launch: %s", cudaGetErrorString(e));
    CK_LAUNCH();
    if (stats) {
        const long long per_plane = partials_per_plane(h);
        lbm::k_reduce_planes<<<h->g.ny, 256, 0, s>>>(h->part, per_plane, h->g.ny, h->acc,
                                                     h->acc + (long long)h->g.ny * lbm::K_STATS);
        CK_LAUNCH();
    }
    return LBM_OK;
}

// One step on stream s; the wall-row launch of a two-launch four-cell step goes
// to s_wall (s when null).
int launch_step(lbm_handle *h, cudaStream_t s, int src, bool stats, cudaStream_t s_wall = nullptr)
{
    if (!s_wall) s_wall = s;
    return h->p.collision == lbm::COLL_MRT ? launch_step_c<lbm::COLL_MRT>(h, s, src, stats, s_wall)
                                           : launch_step_c<lbm::COLL_BGK>(h, s, src, stats, s_wall);
}

// Whether a plain step is the two-launch four-cell form (interior rows, then
// the wall rows with the two-cell tile): both read the source lattice and
// write disjoint rows of the destination, so inside a graph the wall-row
// launch is a parallel branch of the step instead of running after it.
bool two_launch_step(const lbm_handle *h)
{
    return h->kernel == LBM_KERNEL_QUAD && h->layout == LBM_PULL2 && h->g.ny > 2 &&
           (h->p.collision == lbm::COLL_BGK || h->p.wall == lbm::WALL_NODE);
}

int build_chunk(lbm_handle *h, int start)
{
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    const bool fork = LBM_FORK_WALL && two_launch_step(h);
    cudaError_t ce = cudaSuccess;
    for (int i = 0; i < kGraphSteps && rc == LBM_OK && ce == cudaSuccess; ++i) {
        if (fork) {
            // the step's two launches depend on the whole previous step and
            // the next step on both of them
            ce = cudaEventRecord(h->fork, h->cap);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->cap_wall, h->fork, 0);
            if (ce == cudaSuccess) rc = launch_step(h, h->cap, start ^ (i & 1), false, h->cap_wall);
            if (ce == cudaSuccess && rc == LBM_OK) ce = cudaEventRecord(h->join, h->cap_wall);
            if (ce == cudaSuccess && rc == LBM_OK) ce = cudaStreamWaitEvent(h->cap, h->join, 0);
        } else {
            rc = launch_step(h, h->cap, start ^ (i & 1), false);
        }
    }
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (ce != cudaSuccess && rc == LBM_OK) rc = fail(LBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    if (rc != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->chunk[start], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    // move the graph's device-side set-up off its first launch
    e = cudaGraphUpload(h->chunk[start], h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph upload: %s", cudaGetErrorString(e));
    return LBM_OK;
}

// Both chunk graphs (start phase 0 and 1), built together on the first step
// call after any change that invalidated them, whatever the step count, so that
// no capture or instantiation falls inside a later, longer run of steps.
int ensure_chunks(lbm_handle *h)
{
    for (int start = 0; start < 2; ++start)
        if (!h->chunk[start]) {
            const int rc = build_chunk(h, start);
            if (rc != LBM_OK) return rc;
        }
    return LBM_OK;
}

int ensure_part(lbm_handle *h, long long len)
{
    if (len <= h->part_len) return LBM_OK;
    if (h->part) {
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaFree(h->part));
    }
    h->part = nullptr;
    h->part_len = 0;
    if (cudaMalloc((void **)&h->part, len * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "cannot allocate %lld partial sums", len);
    }
    h->part_len = len;
    // the partial buffer is captured by address in the chunk graphs
    for (int i = 0; i < 2; ++i)
        if (h->chunk[i]) {
            cudaGraphExecDestroy(h->chunk[i]);
            h->chunk[i] = nullptr;
        }
    return LBM_OK;
}

int export_state(lbm_handle *h, float *rho, float *u, double *pops, double *part)
{
    const int bx = 128;
    const dim3 grid = grid_of(h, bx);
    const int map = lbm_state_map(h);
    if (h->precision == LBM_FP16_SHIFTED)
        lbm::k_export<__half><<<grid, bx, 0, h->stream>>>((const __half *)lbm_state_ptr(h), h->g, h->p, map, rho, u,
                                                          pops, part);
    else
        lbm::k_export<float><<<grid, bx, 0, h->stream>>>((const float *)lbm_state_ptr(h), h->g, h->p, map, rho, u,
                                                         pops, part);
    CK_LAUNCH();
    return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_last_error(void) { return g_err; }

}  // extern "C"

int lbm_launch_step(lbm_handle *h, cudaStream_t s, int src, bool stats) { return launch_step(h, s, src, stats); }

int lbm_create_handle(lbm_grid g, double tau, double C_s, const double force[3], lbm_wall_model wm, int precision,
                      int layout, void *cuda_stream, void *pop0, void *pop1, lbm_handle **out)
{
    LbmRange range("lbm_create");
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (g.nx < 1 || g.ny < 2 || g.nz < 1) return fail(LBM_ERR_ARG, "grid needs nx >= 1, ny >= 2, nz >= 1");
    if (!(tau > 0.5)) return fail(LBM_ERR_ARG, "tau must exceed 1/2");
    if (!(C_s >= 0.0)) return fail(LBM_ERR_ARG, "C_s must be >= 0");
    if (!force) return fail(LBM_ERR_ARG, "force is NULL");
    if (!isfinite(force[0]) || !isfinite(force[1]) || !isfinite(force[2]))
        return fail(LBM_ERR_ARG, "force must be finite");
    if (wm.kind < LBM_WALL_BB || wm.kind > LBM_WALL_WFB_NODE) return fail(LBM_ERR_ARG, "unknown wall kind");
    if (wm.kind == LBM_WALL_WFB_NODE && g.ny < 3) return fail(LBM_ERR_ARG, "wall nodes need ny >= 3");
    if (wm.kind == LBM_WALL_WFB_NODE && layout == LBM_AA)
        return fail(LBM_ERR_ARG, "wall nodes read the first fluid layer of the source lattice: two-lattice layout only");
    if (wm.law < LBM_LAW_SPALDING || wm.law > LBM_LAW_POWER) return fail(LBM_ERR_ARG, "unknown wall law");
    if (wm.law == LBM_LAW_LOG && !(wm.kappa > 0.0 && wm.B > (1.0 + log(wm.kappa)) / wm.kappa))
        return fail(LBM_ERR_ARG, "log law: y+ and ln(y+)/kappa + B never cross for these kappa, B");
    if ((wm.kind == LBM_WALL_WFB || wm.kind == LBM_WALL_WFB_NODE) && !(wm.kappa > 0.0 && wm.y1 > 0.0))
        return fail(LBM_ERR_ARG, "WFB needs kappa > 0 and y1 > 0");
    if (precision != LBM_FP32 && precision != LBM_FP16_SHIFTED) return fail(LBM_ERR_ARG, "unknown precision");
    if (layout != LBM_PULL2 && layout != LBM_AA) return fail(LBM_ERR_ARG, "unknown layout");
    if (pop0 && layout == LBM_PULL2 && !pop1) return fail(LBM_ERR_ARG, "the two-lattice layout needs two buffers");
    if (pop0 && layout == LBM_AA && pop1) return fail(LBM_ERR_ARG, "the AA layout takes one buffer (pop1 NULL)");
    if ((pop0 && ((uintptr_t)pop0 & 15)) || (pop1 && ((uintptr_t)pop1 & 15)))
        return fail(LBM_ERR_ARG, "population buffers must be 16-byte aligned");
    const int sx = (g.nx + 31) / 32 * 32;
    const long long plane = (long long)sx * g.ny * g.nz;
    if (plane > 2147483647LL) return fail(LBM_ERR_ARG, "grid too large (row-padded cells > 2^31 - 1)");

    lbm_handle *h = new lbm_handle();
    memset(h, 0, sizeof(*h));
    h->g.nx = g.nx;
    h->g.ny = g.ny;
    h->g.nz = g.nz;
    h->g.sx = sx;
    h->g.plane = plane;
    const double nu = wm.nu > 0.0 ? wm.nu : (tau - 0.5) / 3.0;
    h->p.tau0 = (float)tau;
    h->p.smag = (float)(18.0 * sqrt(2.0) * C_s * C_s);
    h->p.Fx = (float)force[0];
    h->p.Fy = (float)force[1];
    h->p.Fz = (float)force[2];
    h->p.wall = wm.kind;
    h->p.kappa = (float)wm.kappa;
    h->p.B = (float)wm.B;
    h->p.ekb = (float)exp(-wm.kappa * wm.B);
    h->p.y1_over_nu = (float)(wm.y1 / nu);
    h->p.newton_iters = wm.newton_iters > 0 ? wm.newton_iters : 12;
    h->p.law = wm.law;
    h->p.ikappa = (float)(1.0 / wm.kappa);
    h->p.pw_a = (float)pow(8.3, 7.0 / 8.0);
    if (wm.law == LBM_LAW_LOG) {
        // upper crossing of y+ and ln(y+)/kappa + B: the map y -> ln(y)/kappa + B
        // contracts (slope 1/(kappa y) < 1) above 1/kappa, so it descends to the
        // root from any start above it
        double y = 1e6;
        for (int i = 0; i < 400; ++i) y = log(y) / wm.kappa + wm.B;
        h->p.law_r2 = (float)(y * y);
    } else if (wm.law == LBM_LAW_POWER) {
        h->p.law_r2 = (float)pow(8.3, 7.0 / 3.0);   // (8.3^(7/6))^2
    }
    for (int c = 0; c < 3; ++c) h->p.hF[c] = (float)(0.5 * force[c]);
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        const double eF = lbm::ex_of(a) * force[0] + lbm::ey_of(a) * force[1] + lbm::ez_of(a) * force[2];
        h->p.weF[k] = (float)(lbm::w_of(a) * eF);
        h->p.WeF[k] = (float)(36.0 * lbm::w_of(a) * eF);
    }
    h->p.t02 = (float)((double)h->p.tau0 * (double)h->p.tau0);
    h->nu_wall = nu;
    // MRT constants: rates of the ghost groups after d'Humieres et al. (2002),
    // s_e 1.19, s_eps 1.4, s_m 1.98, with s_q 1.99 (linear stability near
    // tau0 = 1/2); the stress and pi moments relax with 1/tau_eff. The device
    // correction of group g is (omega - s_g) c_g times a bracket of pair sums
    // (mrt_ghost_pair), c_g = 19 / |row 1|^2, 1 / |row 2|^2, (10/3) / |row 4|^2,
    // 2 / |row 16|^2 from the basis norms.
    h->p.collision = lbm::COLL_BGK;
    h->p.vd_scale = 0.f;
    {
        const double rate[4] = {1.19, 1.4, 1.99, 1.98};
        const double cg[4] = {19.0 / lbm::mrt_norm(1), 1.0 / lbm::mrt_norm(2), (10.0 / 3.0) / lbm::mrt_norm(4),
                              2.0 / lbm::mrt_norm(16)};
        for (int k = 0; k < 4; ++k) {
            h->p.mrt_a[k] = (float)cg[k];
            h->p.mrt_b[k] = (float)(-rate[k] * cg[k]);
        }
    }
    h->precision = precision;
    h->layout = layout;
    h->stream = (cudaStream_t)cuda_stream;
    h->pair = (g.nx % 2) == 0;
    h->wait_limit = lbm::WAIT_CYCLES;

    auto bail = [&](int rc) {
        lbm_free_handle(h);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap_wall, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "cannot create capture streams"));
    const size_t bytes = (size_t)lbm::Q * plane * elem_size(h);
    h->borrowed = pop0 != nullptr;
    if (h->borrowed) {
        h->f[0] = pop0;
        h->f[1] = pop1;
    }
    for (int i = 0; i < (layout == LBM_AA ? 1 : 2) && !h->borrowed; ++i) {
        if (cudaMalloc(&h->f[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(LBM_ERR_OOM, "cannot allocate %zu bytes of populations", bytes));
        }
        if (cudaMemsetAsync(h->f[i], 0, bytes, h->stream) != cudaSuccess)
            return bail(fail(LBM_ERR_CUDA, "memset failed"));
    }
    const size_t twb = (size_t)4 * g.nx * g.nz * sizeof(float);
    const size_t accb = ((size_t)g.ny * lbm::K_STATS + 2 * lbm::K_WALL) * sizeof(double);
    if (cudaMalloc((void **)&h->tw, twb) != cudaSuccess || cudaMalloc((void **)&h->acc, accb) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ERR_OOM, "cannot allocate wall/statistics buffers"));
    }
    if (cudaMemsetAsync(h->tw, 0, twb, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->acc, 0, accb, h->stream) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "memset failed"));
    if (cudaMalloc((void **)&h->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ERR_OOM, "cannot allocate the error flag"));
    }
    if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return bail(fail(LBM_ERR_CUDA, "memset"));
    int rc = select_kernel(h, LBM_KERNEL_AUTO);
    if (rc != LBM_OK) return bail(rc);
    // partial sums: enough for any kernel form on this grid
    const long long nblk = std::max((long long)((g.nx + 31) / 32) * g.ny * g.nz, 8LL * g.ny * g.nz);
    rc = ensure_part(h, nblk * lbm::K_PART);
    if (rc != LBM_OK) return bail(rc);
    *out = h;
    return LBM_OK;
}

int lbm_apply_les(lbm_handle *h, int collision, double u_tau, double a_plus)
{
    if (collision != lbm::COLL_BGK && collision != lbm::COLL_MRT) return fail(LBM_ERR_ARG, "unknown collision");
    if (!(u_tau >= 0.0) || !(a_plus >= 0.0) || (u_tau > 0.0) != (a_plus > 0.0))
        return fail(LBM_ERR_ARG, "van Driest needs both u_tau > 0 and A+ > 0 (or both 0)");
    h->p.collision = collision;
    h->p.vd_scale = a_plus > 0.0 ? (float)(u_tau / (h->nu_wall * a_plus)) : 0.f;
    return LBM_OK;
}

void lbm_free_handle(lbm_handle *h)
{
    if (!h) return;
    if (h->stream || h->f[0]) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; ++i) {
        if (h->chunk[i]) cudaGraphExecDestroy(h->chunk[i]);
        if (h->f[i] && !h->borrowed) cudaFree(h->f[i]);
    }
    if (h->part) cudaFree(h->part);
    if (h->tw) cudaFree(h->tw);
    if (h->acc) cudaFree(h->acc);
    if (h->err) cudaFree(h->err);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cap_wall) cudaStreamDestroy(h->cap_wall);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    delete h;
}

extern "C" {

int lbm_create(lbm_grid g, double tau, double C_s, const double force[3], lbm_wall_model wm, int precision,
               int layout, void *cuda_stream, lbm_handle **out)
{
    return lbm_create_handle(g, tau, C_s, force, wm, precision, layout, cuda_stream, nullptr, nullptr, out);
}

size_t lbm_population_bytes(lbm_grid g, int precision)
{
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return 0;
    if (precision != LBM_FP32 && precision != LBM_FP16_SHIFTED) return 0;
    const size_t sx = (size_t)(g.nx + 31) / 32 * 32;
    return (size_t)lbm::Q * sx * g.ny * g.nz * (precision == LBM_FP16_SHIFTED ? 2 : 4);
}

int lbm_create_from_buffers(lbm_grid g, double tau, double C_s, const double force[3], lbm_wall_model wm,
                            int precision, int layout, void *cuda_stream, void *pop0, void *pop1, lbm_handle **out)
{
    if (out) *out = nullptr;
    if (!pop0) return fail(LBM_ERR_ARG, "pop0 is NULL");
    return lbm_create_handle(g, tau, C_s, force, wm, precision, layout, cuda_stream, pop0, pop1, out);
}

int lbm_init_channel(lbm_handle *h, const double *u_mean_x, double noise_amp, uint64_t seed)
{
    if (!h || !u_mean_x) return fail(LBM_ERR_ARG, "NULL argument");
    double *um = nullptr;
    const size_t b = (size_t)h->g.ny * sizeof(double);
    if (cudaMallocAsync((void **)&um, b, h->stream) != cudaSuccess) return fail(LBM_ERR_OOM, "profile buffer");
    CK(cudaMemcpyAsync(um, u_mean_x, b, cudaMemcpyHostToDevice, h->stream));
    const dim3 grid = grid_of(h, 128);
    if (h->layout == LBM_AA) h->cur = 0;   // written in the natural phase
    const int map = lbm_state_map(h);
    if (h->precision == LBM_FP16_SHIFTED)
        lbm::k_init_channel<__half><<<grid, 128, 0, h->stream>>>((__half *)lbm_state_ptr(h), h->g, h->p.wall, map, um,
                                                                  noise_amp, seed);
    else
        lbm::k_init_channel<float><<<grid, 128, 0, h->stream>>>((float *)lbm_state_ptr(h), h->g, h->p.wall, map, um,
                                                                 noise_amp, seed);
    CK_LAUNCH();
    CK(cudaFreeAsync(um, h->stream));
    // the host profile must stay valid until the copy has run
    CK(cudaStreamSynchronize(h->stream));
    h->step = 0;
    return LBM_OK;
}

int lbm_set_populations(lbm_handle *h, const double *host_in)
{
    LbmRange range("lbm_set_populations");
    if (!h || !host_in) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t b = (size_t)lbm::Q * h->g.nx * h->g.ny * h->g.nz * sizeof(double);
    double *d = nullptr;
    if (cudaMallocAsync((void **)&d, b, h->stream) != cudaSuccess) return fail(LBM_ERR_OOM, "staging buffer");
    CK(cudaMemcpyAsync(d, host_in, b, cudaMemcpyHostToDevice, h->stream));
    const dim3 grid = grid_of(h, 128);
    if (h->layout == LBM_AA) h->cur = 0;
    const int map = lbm_state_map(h);
    if (h->precision == LBM_FP16_SHIFTED)
        lbm::k_scatter<__half><<<grid, 128, 0, h->stream>>>(d, (__half *)lbm_state_ptr(h), h->g, h->p.wall, map);
    else
        lbm::k_scatter<float><<<grid, 128, 0, h->stream>>>(d, (float *)lbm_state_ptr(h), h->g, h->p.wall, map);
    CK_LAUNCH();
    CK(cudaFreeAsync(d, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->step = 0;
    return LBM_OK;
}

int lbm_populations(lbm_handle *h, double *host_out)
{
    LbmRange range("lbm_populations");
    if (!h || !host_out) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t b = (size_t)lbm::Q * h->g.nx * h->g.ny * h->g.nz * sizeof(double);
    double *d = nullptr;
    if (cudaMallocAsync((void **)&d, b, h->stream) != cudaSuccess) return fail(LBM_ERR_OOM, "staging buffer");
    int rc = export_state(h, nullptr, nullptr, d, nullptr);
    if (rc != LBM_OK) return rc;
    CK(cudaMemcpyAsync(host_out, d, b, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(d, h->stream));
    return check_err(h);
}

int lbm_set_stats_every(lbm_handle *h, int every)
{
    if (!h || every < 0) return fail(LBM_ERR_ARG, "invalid argument");
    h->stats_every = every;
    return LBM_OK;
}

int lbm_step(lbm_handle *h, int n)
{
    LbmRange range("lbm_step");
    if (!h || n < 0) return fail(LBM_ERR_ARG, "invalid argument");
    if (h->member) return fail(LBM_ERR_STATE, "a batch member is advanced by lbm_batch_step");
    if (n > 0) {
        const int rc = ensure_chunks(h);
        if (rc != LBM_OK) return rc;
    }
    while (n > 0) {
        const bool sample = h->stats_every > 0 && (h->step % h->stats_every) == 0;
        if (sample) {
            int rc = launch_step(h, h->stream, h->cur, true);
            if (rc != LBM_OK) return rc;
            h->nsamples += 1;
            h->cur ^= 1;
            h->step += 1;
            n -= 1;
            continue;
        }
        long long run = n;
        if (h->stats_every > 0) {
            const long long to_next = h->stats_every - (h->step % h->stats_every);
            if (to_next < run) run = to_next;
        }
        while (run >= kGraphSteps) {
            CK(cudaGraphLaunch(h->chunk[h->cur], h->stream));
            h->step += kGraphSteps;
            run -= kGraphSteps;
            n -= kGraphSteps;
        }
        while (run > 0) {
            int rc = launch_step(h, h->stream, h->cur, false);
            if (rc != LBM_OK) return rc;
            h->cur ^= 1;
            h->step += 1;
            run -= 1;
            n -= 1;
        }
    }
    return LBM_OK;
}

long long lbm_get_step(lbm_handle *h) { return h ? h->step : -1; }

int lbm_set_kernel(lbm_handle *h, int kernel)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (h->member) return fail(LBM_ERR_STATE, "a batch member runs the batch kernel");
    CK(cudaStreamSynchronize(h->stream));
    return select_kernel(h, kernel);
}

int lbm_get_kernel(lbm_handle *h) { return h ? h->kernel : -1; }

int lbm_autotune(lbm_handle *h, int steps, double *best_ms, int *best_kernel)
{
    LbmRange range("lbm_autotune");
    if (!h || steps < 1) return fail(LBM_ERR_ARG, "invalid argument");
    if (h->member) return fail(LBM_ERR_STATE, "a batch member is tuned through its batch");
    CK(cudaStreamSynchronize(h->stream));
    const int forms[4] = {LBM_KERNEL_CELL, LBM_KERNEL_PAIR, LBM_KERNEL_TMA, LBM_KERNEL_QUAD};
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    int best = -1, rc = LBM_OK;
    float best_t = 0.f;
    for (int i = 0; i < 4 && rc == LBM_OK; ++i) {
        if (select_kernel(h, forms[i]) != LBM_OK) continue;   // the grid does not allow this form
        rc = lbm_step(h, 2);                                     // builds the form's graphs
        if (rc != LBM_OK) break;
        float t = 0.f;
        cudaError_t e = cudaEventRecord(ev[0], h->stream);
        if (e == cudaSuccess) rc = lbm_step(h, steps);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventRecord(ev[1], h->stream);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (e != cudaSuccess) rc = fail(LBM_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
        if (rc == LBM_OK) rc = check_err(h);
        if (rc == LBM_OK && (best < 0 || t < best_t)) {
            best = forms[i];
            best_t = t;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != LBM_OK) return rc;
    if (best < 0) return fail(LBM_ERR_ARG, "no kernel form applies to this grid");
    rc = select_kernel(h, best);
    if (rc != LBM_OK) return rc;
    if (best_ms) *best_ms = best_t / steps;
    if (best_kernel) *best_kernel = best;
    return LBM_OK;
}

int lbm_set_les(lbm_handle *h, int collision, double u_tau_ref, double a_plus)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (h->member) return fail(LBM_ERR_STATE, "set the LES model of a batch with lbm_batch_set_les");
    CK(cudaStreamSynchronize(h->stream));
    const int rc = lbm_apply_les(h, collision, u_tau_ref, a_plus);
    if (rc != LBM_OK) return rc;
    return select_kernel(h, h->kernel);   // launch shapes and graphs depend on the operator
}

int lbm_moments(lbm_handle *h, float *rho, float *u, int on_device)
{
    LbmRange range("lbm_moments");
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (!rho && !u) return LBM_OK;
    if (on_device) return export_state(h, rho, u, nullptr, nullptr);
    const long long n = (long long)h->g.nx * h->g.ny * h->g.nz;
    float *d = nullptr;
    if (cudaMallocAsync((void **)&d, (size_t)4 * n * sizeof(float), h->stream) != cudaSuccess)
        return fail(LBM_ERR_OOM, "staging buffer");
    int rc = export_state(h, d, d + n, nullptr, nullptr);
    if (rc != LBM_OK) return rc;
    if (rho) CK(cudaMemcpyAsync(rho, d, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (u) CK(cudaMemcpyAsync(u, d + n, (size_t)3 * n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(d, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_wall_stress(lbm_handle *h, float *tau, int on_device)
{
    if (!h || !tau) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t b = (size_t)4 * h->g.nx * h->g.nz * sizeof(float);
    CK(cudaMemcpyAsync(tau, h->tw, b, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!on_device) CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_plane_stats(lbm_handle *h, double *out, double *wall_out, long long *n_samples, int reset)
{
    LbmRange range("lbm_plane_stats");
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    const size_t b = (size_t)h->g.ny * lbm::K_STATS * sizeof(double);
    if (out) CK(cudaMemcpyAsync(out, h->acc, b, cudaMemcpyDeviceToHost, h->stream));
    if (wall_out)
        CK(cudaMemcpyAsync(wall_out, h->acc + (size_t)h->g.ny * lbm::K_STATS, 2 * lbm::K_WALL * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (n_samples) *n_samples = h->nsamples;
    if (reset) {
        CK(cudaMemsetAsync(h->acc, 0, b + 2 * lbm::K_WALL * sizeof(double), h->stream));
        h->nsamples = 0;
    }
    return LBM_OK;
}

int lbm_conservation(lbm_handle *h, double *out)
{
    LbmRange range("lbm_conservation");
    if (!h || !out) return fail(LBM_ERR_ARG, "NULL argument");
    const dim3 grid = grid_of(h, 128);
    const long long nblk = (long long)grid.x * grid.y * grid.z;
    double *d = nullptr;
    if (cudaMallocAsync((void **)&d, (size_t)(nblk * 4 + 4) * sizeof(double), h->stream) != cudaSuccess)
        return fail(LBM_ERR_OOM, "conservation buffer");
    int rc = export_state(h, nullptr, nullptr, nullptr, d);
    if (rc != LBM_OK) return rc;
    lbm::k_reduce_all<<<1, 256, 0, h->stream>>>(d, nblk, d + nblk * 4);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(out, d + nblk * 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(d, h->stream));
    rc = check_err(h);
    if (rc != LBM_OK) return rc;
    // the partials are deviations from the rest state: add sum w = 1 per cell
    out[0] += (double)h->g.nx * h->g.ny * h->g.nz;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(out[k])) return fail(LBM_ERR_DIVERGED, "non-finite conservation sum (component %d)", k);
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_handle *h, long long cycles)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    h->wait_limit = cycles > 0 ? cycles : lbm::WAIT_CYCLES;
    // captured graphs hold the old limit
    for (int i = 0; i < 2; ++i)
        if (h->chunk[i]) {
            cudaGraphExecDestroy(h->chunk[i]);
            h->chunk[i] = nullptr;
        }
    return LBM_OK;
}

int lbm_sync(lbm_handle *h)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    return check_err(h);
}

void lbm_destroy(lbm_handle *h)
{
    if (!h || h->member) return;   // members are freed with their batch
    lbm_free_handle(h);
}

}  // extern "C"
