// Plane profile of the current state without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want a
// measurement: code that runs while another component owns the allocator (a
// fixed memory budget, a pool that must not grow), host loops that have to
// stay free of allocation calls because those synchronise the device, or
// real-time drivers that forbid allocation after start-up. lbm_plane_profile
// needs block partial sums (scratch), which the rest of the library takes from
// cudaMallocAsync. Here the scratch is a file-scope __device__ array of fixed
// size instead, so the call allocates nothing.
#include <mutex>

#include "lbm.h"
#include "lbm_handle.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int kMaxNy = 2048;        // largest ny the fixed scratch holds
constexpr int kBlocksPerPlane = 8;  // partial sums per wall-normal plane
constexpr int kMaxDevices = 64;

// Block partials [ny][kBlocksPerPlane][K_STATS]: 1.44 MB, held by every GPU
// that loads the library until the process exits. Every call overwrites the
// entries it uses (nothing is accumulated in place), so no clearing is needed;
// two calls whose kernels overlap on the GPU (different streams or handles)
// race on this array.
static __device__ __align__(256) double g_profile_scratch[kMaxNy * kBlocksPerPlane * lbm::K_STATS];

std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code
// g_profile_scratch names a host-side stand-in, not device memory, so the
// address is looked up once per device (with that device current).
int scratch_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm_record_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return lbm_record_error(LBM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_profile_scratch);
        if (e != cudaSuccess || !p) return lbm_record_error(LBM_ERR_CUDA, "cudaGetSymbolAddress of the profile scratch failed");
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

// Per-plane partial sums of rho, u, u u and rho u of the gathered state f(t):
// block (b, y) covers the cells of plane y with z = b, b + 8, ...
template <typename T>
__global__ void __launch_bounds__(256) k_profile_partials(const T *__restrict__ src, lbm::Geom g, lbm::Phys p,
                                                         int map, double *__restrict__ scratch)
{
    const int y = blockIdx.y;
    double v[lbm::K_STATS];
#pragma unroll
    for (int k = 0; k < lbm::K_STATS; ++k) v[k] = 0.0;
    for (int z = blockIdx.x; z < g.nz; z += kBlocksPerPlane) {
        for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
            float f[lbm::Q];
            lbm::gather_any<T>(src, g, p.wall, map, x, y, z, f);
            const lbm::CellState c = lbm::velocity(lbm::moments_of(f), p);
            const double r = c.rho, ux = c.ux, uy = c.uy, uz = c.uz;
            v[0] += r;
            v[1] += ux;
            v[2] += uy;
            v[3] += uz;
            v[4] += ux * ux;
            v[5] += uy * uy;
            v[6] += uz * uz;
            v[7] += ux * uy;
            v[8] += r * ux;
            v[9] += r * uy;
            v[10] += r * uz;
        }
    }
    lbm::block_reduce_store<lbm::K_STATS>(v, scratch + ((long long)y * kBlocksPerPlane + blockIdx.x) * lbm::K_STATS);
}

__global__ void k_profile_finish(const double *__restrict__ scratch, int ny, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ny * lbm::K_STATS) return;
    const int y = i / lbm::K_STATS, k = i % lbm::K_STATS;
    double s = 0.0;
    for (int b = 0; b < kBlocksPerPlane; ++b) s += scratch[((long long)y * kBlocksPerPlane + b) * lbm::K_STATS + k];
    out[i] = s;
}

}  // namespace

extern "C" int lbm_plane_profile_noalloc(lbm_handle *h, double *out_dev)
{
    if (!h || !out_dev) return lbm_record_error(LBM_ERR_ARG, "NULL argument");
    if (h->g.ny > kMaxNy)
        return lbm_record_error(LBM_ERR_ARG,
                                "lbm_plane_profile_noalloc: ny exceeds the fixed scratch limit of 2048 planes");
    double *scratch = nullptr;
    const int rc = scratch_on_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    const dim3 grid(kBlocksPerPlane, h->g.ny);
    if (h->precision == LBM_FP16_SHIFTED)
        k_profile_partials<__half><<<grid, 256, 0, h->stream>>>((const __half *)lbm_state_ptr(h), h->g, h->p,
                                                                lbm_state_map(h), scratch);
    else
        k_profile_partials<float><<<grid, 256, 0, h->stream>>>((const float *)lbm_state_ptr(h), h->g, h->p,
                                                               lbm_state_map(h), scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lbm_record_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    const int n = h->g.ny * lbm::K_STATS;
    k_profile_finish<<<(n + 255) / 256, 256, 0, h->stream>>>(scratch, h->g.ny, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return lbm_record_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}
