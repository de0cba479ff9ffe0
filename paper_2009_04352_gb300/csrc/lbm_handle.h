// Internal layout of an lbm_handle, shared by the translation units of the
// library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_device.cuh"

struct lbm_handle {
    lbm::Geom g;
    lbm::Phys p;
    int precision;
    int layout;
    cudaStream_t stream;
    cudaStream_t cap;            // private stream used only for graph capture
    cudaStream_t cap_wall;       // second capture stream: the wall-row branch of a four-cell step
    cudaEvent_t fork, join;      // fork and join of that branch inside a capture
    void *f[2];                  // two lattices (AA: f[0] only)
    int cur;                     // PULL2: lattice holding the current state; AA: phase (0 or 1)
    long long step;
    int stats_every;
    float *tw;                   // [2][nz][nx][2]
    double *part;                // block partials
    long long part_len;          // doubles
    double *acc;                 // [ny][K_STATS] then [2][K_WALL]
    long long nsamples;
    int bx;                      // threads per block along x (one-cell / two-cell kernels)
    bool pair;                   // two cells per thread (even nx)
    int kernel;                  // LBM_KERNEL_* in use (never AUTO)
    int tma_grid;                // CTAs of the row-pipelined kernel
    int tma_warps;               // warps per CTA of the row-pipelined kernel (4 or 8)
    int tma_stages;              // ring stages of the row-pipelined kernel
    int tma_smem;                // dynamic shared memory bytes of the row-pipelined kernel
    int *err;                    // device flag set by a timed-out pipeline wait
    long long wait_limit;        // clock cycles a pipeline wait may take before it gives up
    cudaGraphExec_t chunk[2];    // kGraphSteps plain steps starting from cur = 0 / 1
    bool member;                 // member view of a batch (stepped by the batch)
    bool borrowed;               // population arrays owned by the caller or a batch, not freed here
    double nu_wall;              // viscosity of the wall law and of the van Driest y+
};

// The array holding the current state and the map under which f(t) is stored.
inline void *lbm_state_ptr(const lbm_handle *h) { return h->layout == LBM_AA ? h->f[0] : h->f[h->cur]; }
inline int lbm_state_map(const lbm_handle *h)
{
    if (h->layout != LBM_AA) return lbm::MAP_PULL;
    return h->cur ? lbm::MAP_AA1 : lbm::MAP_AA0;
}

// Set the LES model of a handle's physics: collision (COLL_BGK / COLL_MRT)
// and the van Driest factor (u_tau > 0 and a_plus > 0, else no damping).
int lbm_apply_les(lbm_handle *h, int collision, double u_tau, double a_plus);

// Create a handle; with pop0 non-NULL its population arrays are borrowed
// (a batch pool or caller buffers; nothing is allocated or freed for them).
// pop1 is the second lattice of the two-lattice layout (NULL for AA).
int lbm_create_handle(lbm_grid g, double tau, double C_s, const double force[3], lbm_wall_model wm, int precision,
                      int layout, void *cuda_stream, void *pop0, void *pop1, lbm_handle **out);

// Free a handle, member views included.
void lbm_free_handle(lbm_handle *h);

// Launch one step of a handle's own kernels on stream s from state `src`
// (lattice, or AA phase), plane statistics fused when `stats`.
int lbm_launch_step(lbm_handle *h, cudaStream_t s, int src, bool stats);

// Record an error message for lbm_last_error() and return `code`.
int lbm_record_error(int code, const char *msg);

// Host-side NVTX range over one library call (visible in Nsight timelines; a
// no-op without a profiler attached).
struct LbmRange {
    explicit LbmRange(const char *name) { nvtxRangePushA(name); }
    ~LbmRange() { nvtxRangePop(); }
    LbmRange(const LbmRange &) = delete;
    LbmRange &operator=(const LbmRange &) = delete;
};
