// ucp_static.cu -- an entry point that allocates no device memory: the
// enclosing-cube reduction (the first step of the TREE construction) with its
// per-tile partial results kept in a fixed, file-scope device array.
#include "ucp.h"
#include "ucp_internal.cuh"

#include <cuda.h>
#include <cuda_runtime.h>

#include <math.h>

#include <mutex>

namespace {

constexpr int kTile = UCP_STATIC_TILE;        // particles reduced by one block
constexpr int kMaxTiles = UCP_STATIC_MAX_N / UCP_STATIC_TILE;
constexpr int kThreads = 256;

// Scratch for the per-tile {min xyz, max xyz} (ordered integer images of the
// doubles); every GPU that loads the library holds one copy (48 KB) until the
// process exits.
static __device__ __align__(256) unsigned long long g_cube_scratch[kMaxTiles * 6];

// Device address of g_cube_scratch per device, with the CUDA context it was
// looked up in: a device reset or a new primary context makes a new lookup.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    void* ctx;
    unsigned long long* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

// Min and max of each axis as ordered integer images (ord64): the reductions of
// the library's own cube (k_bbox_partial, k_bbox_final), so the two cubes agree
// for every input, signed zeros and NaN included.
__global__ void __launch_bounds__(kThreads)
k_cube_tiles(const double* __restrict__ pos, int n, unsigned long long* __restrict__ part)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    const int b = blockIdx.x * kTile, e = min(n, b + kTile);
    for (int i = b + threadIdx.x; i < e; i += kThreads)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long v = ucp::ord64(pos[3 * (size_t)i + a]);
            lo[a] = min(lo[a], v);
            hi[a] = max(hi[a], v);
        }
    __shared__ unsigned long long s[kThreads][6];
    for (int a = 0; a < 3; ++a) {
        s[threadIdx.x][a] = lo[a];
        s[threadIdx.x][3 + a] = hi[a];
    }
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int a = 0; a < 3; ++a) {
                s[threadIdx.x][a] = min(s[threadIdx.x][a], s[threadIdx.x + st][a]);
                s[threadIdx.x][3 + a] = max(s[threadIdx.x][3 + a], s[threadIdx.x + st][3 + a]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[0][threadIdx.x];
}

// Same cube as the library's tree build: centre (min + max) / 2, side = largest
// extent * (1 + 2^-20), side 1 when every particle coincides.
__global__ void __launch_bounds__(kThreads)
k_cube_final(const unsigned long long* __restrict__ part, int ntiles, double* __restrict__ out)
{
    __shared__ unsigned long long s[kThreads][6];
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int b = threadIdx.x; b < ntiles; b += kThreads)
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], part[6 * b + a]);
            hi[a] = max(hi[a], part[6 * b + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) {
        s[threadIdx.x][a] = lo[a];
        s[threadIdx.x][3 + a] = hi[a];
    }
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int a = 0; a < 3; ++a) {
                s[threadIdx.x][a] = min(s[threadIdx.x][a], s[threadIdx.x + st][a]);
                s[threadIdx.x][3 + a] = max(s[threadIdx.x][3 + a], s[threadIdx.x + st][3 + a]);
            }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double mn = ucp::unord64(s[0][a]), mx = ucp::unord64(s[0][3 + a]);
        out[a] = __dmul_rn(__dadd_rn(mn, mx), 0.5);
        double e = __dsub_rn(mx, mn);
        if (e > ext) ext = e;
    }
    out[3] = ext > 0.0 ? __dmul_rn(ext, 1.0 + 0x1p-20) : 1.0;
}

}  // namespace

extern "C" int ucp_root_cube_static(const double* pos, int64_t n, double* cube_out, void* stream)
{
    if (!pos || !cube_out) return UCP_EINVAL;
    if (n < 1 || n > (int64_t)UCP_STATIC_MAX_N) return UCP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return UCP_ECUDA;
    unsigned long long* scratch;
    {
        std::lock_guard<std::mutex> g(g_scratch_mu);
        if (!g_ctx_get_current) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault,
                                                 &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn) {
                cudaGetLastError();
                return UCP_ECUDA;
            }
            g_ctx_get_current = (CtxGetCurrentFn)fn;
        }
        CUcontext ctx = nullptr;
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return UCP_ECUDA;
        if (!g_scratch[dev].ptr || g_scratch[dev].ctx != (void*)ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_cube_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return UCP_ECUDA;
            }
            if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return UCP_ECUDA;
            g_scratch[dev].ptr = (unsigned long long*)p;
            g_scratch[dev].ctx = (void*)ctx;
        }
        scratch = g_scratch[dev].ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int ntiles = (int)((n + kTile - 1) / kTile);
    ucp::count_launch(2);
    k_cube_tiles<<<ntiles, kThreads, 0, s>>>(pos, (int)n, scratch);
    k_cube_final<<<1, kThreads, 0, s>>>(scratch, ntiles, cube_out);
    return cudaGetLastError() == cudaSuccess ? UCP_OK : UCP_ECUDA;
}
