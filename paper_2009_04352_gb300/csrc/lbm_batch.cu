// Batched ensemble: many independent channels of uneven sizes and parameters
// advanced together, each step replayed from CUDA graphs. Two forms:
//
// * Persistent form: ONE persistent kernel launch per time step. All members'
//   lattices live in one device pool. The work list is the concatenation of
//   every member's tiles (a tile = 2 * threads consecutive cells of one (y, z)
//   row, the unit of the two-cell kernel); member i owns tiles [tile0_i,
//   tile0_i + tiles_i). A grid of CTAs sized to the GPU (CTAs per SM x SM
//   count) splits the list into contiguous shares; a CTA finds the member of
//   its first tile by binary search over tile0, stages the member's descriptor
//   (geometry, physics, pool offsets) in shared memory, and then advances
//   (tile, row, member) incrementally, running the same tile code as the
//   single-channel kernel.
// * Member-grid form: every member runs the single-channel step kernels its
//   own grid selects (four-cell for FP16 storage, two-cell for FP32), with
//   its geometry and physics as launch parameters; the members are spread
//   over a few capture streams balanced by cell count and each 16-step chunk
//   of all members is captured as one CUDA graph, so the members' grids run
//   concurrently and small members fill the gaps of large ones.
//
// Sampled steps add one plane reduction per member. The form and its launch
// shape (threads per CTA and CTAs per SM, or streams) are chosen by a timing
// autotuner.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lbm.h"
#include "lbm_handle.h"
#include "lbm_pair.cuh"

namespace {

constexpr int kBatchGraphSteps = 16;
constexpr int kMaxStreams = 32;   // capture streams of the member-grid form

struct BatchInst {
    lbm::Geom g;
    lbm::Phys p;
    long long off[2];   // element offsets of the member's two lattices in the pool
    float *tw;          // member's wall-stress plane
    double *part;       // member's block partials
    long long tile0;    // first tile of the member
    int nxb;            // tiles per row
};

#ifndef LBM_BATCH_MIN_BLOCKS
#define LBM_BATCH_MIN_BLOCKS 5   // resident CTAs per SM the register budget must allow
#endif

template <typename T, bool STATS, int COLL>
__global__ void __launch_bounds__(128, LBM_BATCH_MIN_BLOCKS) k_batch_step(const BatchInst *__restrict__ inst, int n, long long total,
                                                    T *__restrict__ pool, int cur)
{
    lbm::pdl_begin();
    // this CTA's contiguous share [t, t1) of the work list
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    long long t = (long long)blockIdx.x * per;
    const long long t1 = t + per < total ? t + per : total;
    if (t >= t1) return;
    __shared__ BatchInst s;
    int m = 0;   // last member whose first tile is <= t
    {
        int hi = n - 1;
        while (m < hi) {
            const int mid = (m + hi + 1) >> 1;
            if (inst[mid].tile0 <= t)
                m = mid;
            else
                hi = mid - 1;
        }
    }
    if (threadIdx.x == 0) s = inst[m];
    __syncthreads();
    // position of tile t inside member m, then advanced tile by tile
    int xb, y, z;
    {
        const long long local = t - s.tile0;
        xb = (int)(local % s.nxb);
        const long long row = local / s.nxb;
        y = (int)(row % s.g.ny);
        z = (int)(row / s.g.ny);
    }
    for (;;) {
        double *part = STATS ? s.part + (((long long)y * s.g.nz + z) * s.nxb + xb) * lbm::K_PART : nullptr;
        if constexpr (sizeof(T) == 2) {
            // FP16 storage: interior rows run an instantiation without
            // wall-layer code (+7% measured; FP32, DRAM-bound, loses 2% with it)
            if (y == 0 || y == s.g.ny - 1)
                lbm::pair_tile<T, STATS, COLL, lbm::LAY_PULL, lbm::ROWS_WALL>(pool + s.off[cur], pool + s.off[cur ^ 1],
                                                                             s.g, s.p, s.tw, part, xb, y, z);
            else
                lbm::pair_tile<T, STATS, COLL, lbm::LAY_PULL, lbm::ROWS_INTERIOR>(
                    pool + s.off[cur], pool + s.off[cur ^ 1], s.g, s.p, s.tw, part, xb, y, z);
        } else {
            lbm::pair_tile<T, STATS, COLL>(pool + s.off[cur], pool + s.off[cur ^ 1], s.g, s.p, s.tw, part, xb, y, z);
        }
        if (++t >= t1) break;
        if (++xb == s.nxb) {
            xb = 0;
            if (++y == s.g.ny) {
                y = 0;
                if (++z == s.g.nz) {
                    z = 0;
                    ++m;   // next member: every thread reaches this point together
                    __syncthreads();
                    if (threadIdx.x == 0) s = inst[m];
                    __syncthreads();
                }
            }
        }
    }
}

int fail(int code, const char *msg) { return lbm_record_error(code, msg); }

int fail_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return lbm_record_error(LBM_ERR_CUDA, buf);
}

#define BK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
    } while (0)

}  // namespace

struct lbm_batch {
    int n;
    int precision;
    cudaStream_t stream;
    cudaStream_t cap;
    std::vector<lbm_handle *> members;
    void *pool;
    std::vector<long long> off;   // per member: offset of lattice 0 (lattice 1 follows)
    BatchInst *d_inst;
    long long tiles;
    int form;                     // LBM_BATCH_PERSISTENT or LBM_BATCH_MEMBER_GRIDS
    int threads;                  // threads per CTA (tile = 2 * threads cells)
    int ctas_per_sm;
    int grid;
    int sms;
    int nstreams;                 // member-grid form: capture streams in use
    cudaStream_t side[kMaxStreams];
    cudaEvent_t fork, join[kMaxStreams];
    std::vector<int> lane;        // member-grid form: capture stream of each member
    int cur;
    long long step;
    int stats_every;
    cudaGraphExec_t chunk[2];
};

namespace {

size_t elem_bytes(int precision) { return precision == LBM_FP16_SHIFTED ? 2 : 4; }

void drop_graphs(lbm_batch *b)
{
    for (int i = 0; i < 2; ++i)
        if (b->chunk[i]) {
            cudaGraphExecDestroy(b->chunk[i]);
            b->chunk[i] = nullptr;
        }
}

template <typename T, int COLL>
int occupancy_c(int threads, int *out)
{
    int per_sm = 0, st = 0;
    BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<T, false, COLL>, threads, 0));
    BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&st, k_batch_step<T, true, COLL>, threads, 0));
    *out = std::min(per_sm, st);
    return LBM_OK;
}

int max_ctas_per_sm(const lbm_batch *b, int threads, int *out)
{
    const bool mrt = b->members[0]->p.collision == lbm::COLL_MRT;
    if (b->precision == LBM_FP16_SHIFTED)
        return mrt ? occupancy_c<__half, lbm::COLL_MRT>(threads, out) : occupancy_c<__half, lbm::COLL_BGK>(threads, out);
    return mrt ? occupancy_c<float, lbm::COLL_MRT>(threads, out) : occupancy_c<float, lbm::COLL_BGK>(threads, out);
}

// Rebuild the descriptor table for `threads` per CTA and size the grid.
int configure(lbm_batch *b, int threads, int ctas_per_sm)
{
    if (threads != 64 && threads != 128) return fail(LBM_ERR_ARG, "threads per CTA must be 64 or 128");
    int max_per_sm = 0;
    int rc = max_ctas_per_sm(b, threads, &max_per_sm);
    if (rc != LBM_OK) return rc;
    if (ctas_per_sm <= 0 || ctas_per_sm > max_per_sm) ctas_per_sm = max_per_sm;
    std::vector<BatchInst> h(b->n);
    long long tile = 0;
    for (int i = 0; i < b->n; ++i) {
        const lbm_handle *m = b->members[i];
        BatchInst &d = h[i];
        memset(&d, 0, sizeof(d));
        d.g = m->g;
        d.p = m->p;
        d.off[0] = b->off[i];
        d.off[1] = b->off[i] + (long long)lbm::Q * m->g.plane;
        d.tw = m->tw;
        d.part = m->part;
        d.nxb = (m->g.nx / 2 + threads - 1) / threads;
        d.tile0 = tile;
        tile += (long long)d.nxb * m->g.ny * m->g.nz;
    }
    BK(cudaStreamSynchronize(b->stream));
    BK(cudaMemcpy(b->d_inst, h.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice));
    b->tiles = tile;
    b->threads = threads;
    b->ctas_per_sm = ctas_per_sm;
    b->grid = (int)std::min<long long>((long long)b->sms * ctas_per_sm, tile);
    drop_graphs(b);
    return LBM_OK;
}

template <typename T, bool STATS, int COLL>
cudaError_t launch_pdl(lbm_batch *b, cudaStream_t s, int cur)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(b->threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    // FP32 tiles read the source lattice through the read-only path, which
    // rules out starting while the previous step drains (pull_nc)
    attr[0].val.programmaticStreamSerializationAllowed = lbm::pull_nc<T> ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_step<T, STATS, COLL>, (const BatchInst *)b->d_inst, b->n, b->tiles,
                              (T *)b->pool, cur);
}

// Member-grid form: spread the members over `streams` capture streams,
// largest first onto the least loaded.
void assign_streams(lbm_batch *b, int streams)
{
    b->nstreams = streams;
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    auto cells = [&](int i) { return (long long)b->members[i]->g.nx * b->members[i]->g.ny * b->members[i]->g.nz; };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cells(x) > cells(y); });
    std::vector<long long> load(streams, 0);
    b->lane.assign(b->n, 0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->lane[i] = k;
        load[k] += cells(i);
    }
}

int launch(lbm_batch *b, cudaStream_t s, int cur, bool stats)
{
    if (b->form == LBM_BATCH_MEMBER_GRIDS) {
        // one member after the other on s (the graphs of plain steps run the
        // members on their capture streams instead)
        for (lbm_handle *m : b->members) {
            const int rc = lbm_launch_step(m, s, cur, stats);
            if (rc != LBM_OK) return rc;
        }
        return LBM_OK;
    }
    cudaError_t e;
    const bool mrt = b->members[0]->p.collision == lbm::COLL_MRT;
    if (b->precision == LBM_FP16_SHIFTED) {
        if (mrt)
            e = stats ? launch_pdl<__half, true, lbm::COLL_MRT>(b, s, cur) : launch_pdl<__half, false, lbm::COLL_MRT>(b, s, cur);
        else
            e = stats ? launch_pdl<__half, true, lbm::COLL_BGK>(b, s, cur) : launch_pdl<__half, false, lbm::COLL_BGK>(b, s, cur);
    } else {
        if (mrt)
            e = stats ? launch_pdl<float, true, lbm::COLL_MRT>(b, s, cur) : launch_pdl<float, false, lbm::COLL_MRT>(b, s, cur);
        else
            e = stats ? launch_pdl<float, true, lbm::COLL_BGK>(b, s, cur) : launch_pdl<float, false, lbm::COLL_BGK>(b, s, cur);
    }
    if (e != cudaSuccess) return fail_cuda(e, "batch step launch");
    if (stats) {
        for (int i = 0; i < b->n; ++i) {
            lbm_handle *m = b->members[i];
            const long long per_plane = (long long)((m->g.nx / 2 + b->threads - 1) / b->threads) * m->g.nz;
            lbm::k_reduce_planes<<<m->g.ny, 256, 0, s>>>(m->part, per_plane, m->g.ny, m->acc,
                                                         m->acc + (long long)m->g.ny * lbm::K_STATS);
        }
        BK(cudaGetLastError());
    }
    return LBM_OK;
}

int build_chunk(lbm_batch *b, int start)
{
    cudaGraph_t graph = nullptr;
    BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    if (b->form == LBM_BATCH_MEMBER_GRIDS) {
        // fork to the capture streams, each runs its members' 16 steps in
        // step order, join
        cudaError_t ce = cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < b->nstreams && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        if (ce != cudaSuccess) rc = fail_cuda(ce, "graph fork");
        for (int i = 0; i < kBatchGraphSteps && rc == LBM_OK; ++i)
            for (int m = 0; m < b->n && rc == LBM_OK; ++m)
                rc = lbm_launch_step(b->members[m], b->side[b->lane[m]], start ^ (i & 1), false);
        for (int k = 0; k < b->nstreams && ce == cudaSuccess; ++k) {
            ce = cudaEventRecord(b->join[k], b->side[k]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->cap, b->join[k], 0);
        }
        if (ce != cudaSuccess && rc == LBM_OK) rc = fail_cuda(ce, "graph join");
    } else {
        for (int i = 0; i < kBatchGraphSteps && rc == LBM_OK; ++i) rc = launch(b, b->cap, start ^ (i & 1), false);
    }
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail_cuda(e, "graph capture");
    e = cudaGraphInstantiate(&b->chunk[start], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(e, "graph instantiate");
    e = cudaGraphUpload(b->chunk[start], b->stream);
    if (e != cudaSuccess) return fail_cuda(e, "graph upload");
    return LBM_OK;
}

// Both chunk graphs, built on the first step call after a reconfiguration
// (whatever its step count), so that no capture lands inside a later run.
int ensure_chunks(lbm_batch *b)
{
    for (int start = 0; start < 2; ++start)
        if (!b->chunk[start]) {
            const int rc = build_chunk(b, start);
            if (rc != LBM_OK) return rc;
        }
    return LBM_OK;
}

void sync_members(lbm_batch *b)
{
    for (lbm_handle *m : b->members) {
        m->cur = b->cur;
        m->step = b->step;
    }
}

}  // namespace

extern "C" {

int lbm_batch_create(int n, const lbm_member *members, int precision, void *cuda_stream, lbm_batch **out)
{
    LbmRange range("lbm_batch_create");
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !members) return fail(LBM_ERR_ARG, "a batch needs n >= 1 members");
    if (precision != LBM_FP32 && precision != LBM_FP16_SHIFTED) return fail(LBM_ERR_ARG, "unknown precision");
    for (int i = 0; i < n; ++i)
        if (members[i].grid.nx < 2 || members[i].grid.nx % 2)
            return fail(LBM_ERR_ARG, "batch members need an even nx >= 2");
    lbm_batch *b = new lbm_batch();
    b->n = n;
    b->precision = precision;
    b->stream = (cudaStream_t)cuda_stream;
    b->chunk[0] = b->chunk[1] = nullptr;
    b->pool = nullptr;
    b->d_inst = nullptr;
    b->cap = nullptr;
    b->fork = nullptr;
    b->nstreams = 0;
    for (int k = 0; k < kMaxStreams; ++k) {
        b->side[k] = nullptr;
        b->join[k] = nullptr;
    }
    auto bail = [&](int rc) {
        lbm_batch_destroy(b);
        return rc;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "cannot query the device"));
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "cannot create capture stream"));
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "cannot create capture events"));
    for (int k = 0; k < kMaxStreams; ++k)
        if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(LBM_ERR_CUDA, "cannot create capture streams"));
    // pool layout: per member two lattices of 19 row-padded planes, 256-byte aligned
    const size_t eb = elem_bytes(precision);
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_grid &g = members[i].grid;
        const long long sx = (g.nx + 31) / 32 * 32;
        const long long plane = sx * g.ny * g.nz;
        if (plane > 2147483647LL) return bail(fail(LBM_ERR_ARG, "a member grid is too large"));
        b->off.push_back(total);
        total += 2LL * lbm::Q * plane;
        total = (total * (long long)eb + 255) / 256 * 256 / (long long)eb;
    }
    if (cudaMalloc(&b->pool, (size_t)total * eb) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ERR_OOM, "cannot allocate the batch population pool"));
    }
    if (cudaMemsetAsync(b->pool, 0, (size_t)total * eb, b->stream) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, "memset failed"));
    for (int i = 0; i < n; ++i) {
        const lbm_member &m = members[i];
        char *base = (char *)b->pool + (size_t)b->off[i] * eb;
        const long long sx = (m.grid.nx + 31) / 32 * 32;
        char *second = base + (size_t)lbm::Q * sx * m.grid.ny * m.grid.nz * eb;
        lbm_handle *h = nullptr;
        const int rc = lbm_create_handle(m.grid, m.tau, m.C_s, m.force, m.wall, precision, LBM_PULL2, cuda_stream, base,
                                         second, &h);
        if (rc != LBM_OK) return bail(rc);
        h->member = true;
        b->members.push_back(h);
    }
    if (cudaMalloc((void **)&b->d_inst, sizeof(BatchInst) * n) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ERR_OOM, "cannot allocate the batch descriptors"));
    }
    b->cur = 0;
    b->step = 0;
    b->stats_every = 0;
    b->form = LBM_BATCH_MEMBER_GRIDS;   // measured faster than the persistent form on GB300
    assign_streams(b, 8);
    const int rc = configure(b, 128, 0);
    if (rc != LBM_OK) return bail(rc);
    *out = b;
    return LBM_OK;
}

lbm_handle *lbm_batch_member(lbm_batch *b, int i)
{
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->members[i];
}

long long lbm_batch_cells(lbm_batch *b)
{
    if (!b) return -1;
    long long c = 0;
    for (const lbm_handle *m : b->members) c += (long long)m->g.nx * m->g.ny * m->g.nz;
    return c;
}

int lbm_batch_set_stats_every(lbm_batch *b, int every)
{
    if (!b || every < 0) return fail(LBM_ERR_ARG, "invalid argument");
    b->stats_every = every;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int n)
{
    LbmRange range("lbm_batch_step");
    if (!b || n < 0) return fail(LBM_ERR_ARG, "invalid argument");
    if (n > 0) {
        const int rc = ensure_chunks(b);
        if (rc != LBM_OK) return rc;
    }
    while (n > 0) {
        const bool sample = b->stats_every > 0 && (b->step % b->stats_every) == 0;
        if (sample) {
            const int rc = launch(b, b->stream, b->cur, true);
            if (rc != LBM_OK) return rc;
            for (lbm_handle *m : b->members) m->nsamples += 1;
            b->cur ^= 1;
            b->step += 1;
            n -= 1;
            continue;
        }
        long long run = n;
        if (b->stats_every > 0) run = std::min<long long>(run, b->stats_every - (b->step % b->stats_every));
        while (run >= kBatchGraphSteps) {
            BK(cudaGraphLaunch(b->chunk[b->cur], b->stream));
            b->step += kBatchGraphSteps;
            run -= kBatchGraphSteps;
            n -= kBatchGraphSteps;
        }
        while (run > 0) {
            const int rc = launch(b, b->stream, b->cur, false);
            if (rc != LBM_OK) return rc;
            b->cur ^= 1;
            b->step += 1;
            run -= 1;
            n -= 1;
        }
    }
    sync_members(b);
    return LBM_OK;
}

int lbm_batch_set_config(lbm_batch *b, int threads, int ctas_per_sm)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    return configure(b, threads, ctas_per_sm);
}

int lbm_batch_get_config(lbm_batch *b, int *threads, int *ctas_per_sm, int *grid, long long *tiles)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    if (threads) *threads = b->threads;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (grid) *grid = b->grid;
    if (tiles) *tiles = b->tiles;
    return LBM_OK;
}

int lbm_batch_set_form(lbm_batch *b, int form, int streams)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    if (form != LBM_BATCH_PERSISTENT && form != LBM_BATCH_MEMBER_GRIDS) return fail(LBM_ERR_ARG, "unknown batch form");
    if (streams < 0 || streams > kMaxStreams) return fail(LBM_ERR_ARG, "streams must be 0 .. 32");
    BK(cudaStreamSynchronize(b->stream));
    b->form = form;
    assign_streams(b, streams == 0 ? 8 : streams);
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_get_form(lbm_batch *b, int *streams)
{
    if (!b) return -1;
    if (streams) *streams = b->nstreams;
    return b->form;
}

int lbm_batch_autotune(lbm_batch *b, int steps, double *best_ms)
{
    LbmRange range("lbm_batch_autotune");
    if (!b || steps < 1) return fail(LBM_ERR_ARG, "invalid argument");
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    double best = 1e300;
    int best_form = LBM_BATCH_PERSISTENT, best_t = 128, best_c = 0, best_s = 8;
    const int saved_stats = b->stats_every;
    b->stats_every = 0;
    auto time_shape = [&](int form, int threads, int c, int streams) -> int {
        b->form = form;
        assign_streams(b, streams);
        int rc = configure(b, threads, c);
        if (rc == LBM_OK) rc = lbm_batch_step(b, 2);   // warm-up (builds the step graphs)
        if (rc != LBM_OK) return rc;
        BK(cudaEventRecord(e0, b->stream));
        rc = lbm_batch_step(b, steps);
        if (rc != LBM_OK) return rc;
        BK(cudaEventRecord(e1, b->stream));
        BK(cudaEventSynchronize(e1));
        float ms = 0.f;
        BK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_form = form;
            best_t = threads;
            best_c = c;
            best_s = streams;
        }
        return LBM_OK;
    };
    for (int threads : {64, 128}) {
        int max_per_sm = 0;
        int rc = max_ctas_per_sm(b, threads, &max_per_sm);
        if (rc != LBM_OK) return rc;
        for (int c = std::max(1, max_per_sm / 4); c <= max_per_sm; c += std::max(1, max_per_sm / 4)) {
            rc = time_shape(LBM_BATCH_PERSISTENT, threads, c, b->nstreams);
            if (rc != LBM_OK) return rc;
        }
    }
    for (int streams : {4, 8, 16}) {
        const int rc = time_shape(LBM_BATCH_MEMBER_GRIDS, b->threads, b->ctas_per_sm, std::min(streams, b->n));
        if (rc != LBM_OK) return rc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->stats_every = saved_stats;
    if (best_ms) *best_ms = best / steps;
    b->form = best_form;
    assign_streams(b, best_s);
    return configure(b, best_t, best_c);
}

int lbm_batch_set_les(lbm_batch *b, int collision, const double *u_tau_ref, double a_plus)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    BK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        const double ut = u_tau_ref ? u_tau_ref[i] : 0.0;
        const int rc = lbm_apply_les(b->members[i], collision, ut, ut > 0.0 ? a_plus : 0.0);
        if (rc != LBM_OK) return rc;
    }
    return configure(b, b->threads, b->ctas_per_sm);   // descriptors carry the physics
}

int lbm_batch_sync(lbm_batch *b)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    BK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (int k = 0; k < kMaxStreams; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    for (lbm_handle *m : b->members) lbm_free_handle(m);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->pool) cudaFree(b->pool);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
