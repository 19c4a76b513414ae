// ucp_schedule.cu -- order of the walk's work: after each walk the chunk list
// of its targets is rewritten longest-first by the cost each chunk just had
// (20 per direct pair + 64 per multipole, summed over its targets), so the next
// walk over the same targets (the next substep) starts the expensive chunks first
// and the persistent grid does not end on a few long ones.  The order of chunks
// changes no result: every warp walks whole chunks.
#include "ucp_internal.cuh"

namespace ucp {

namespace {

// ---- walk schedule: chunks in decreasing order of their last measured cost
// (longest first), so the persistent grid does not end on a few long chunks.
// The order of chunks changes no result.
__global__ void __launch_bounds__(256)
k_chunk_cost(const int4* __restrict__ chunks, int nchunks, const int* __restrict__ targets,
             const int* __restrict__ cnt_p2p, const int* __restrict__ cnt_m2p,
             float* __restrict__ cost)
{
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nchunks) return;
    const int4 ck = chunks[w];
    float v = 0.f;
    if (lane < ck.y) {
        const int ti = ck.x + lane;
        const int t = targets ? targets[ti] : ti;
        v = 20.f * (float)cnt_p2p[t] + 64.f * (float)cnt_m2p[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) cost[w] = v;
}

constexpr int kLptThreads = 1024;
constexpr int kLptBins = 256;

// One block: bin the chunks by cost / max cost, then place them bin by bin from
// the most expensive; the chunk list is rewritten in that order.
__global__ void __launch_bounds__(kLptThreads)
k_chunk_lpt(int4* __restrict__ chunks, int nchunks, const float* __restrict__ cost,
            int4* __restrict__ tmp)
{
    __shared__ int hist[kLptBins];
    __shared__ float red[kLptThreads / 32];
    float mx = 0.f;
    for (int i = threadIdx.x; i < nchunks; i += kLptThreads) mx = fmaxf(mx, cost[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    for (int b = threadIdx.x; b < kLptBins; b += kLptThreads) hist[b] = 0;
    __syncthreads();
    mx = 0.f;
    for (int k = 0; k < kLptThreads / 32; ++k) mx = fmaxf(mx, red[k]);
    const float scale = mx > 0.f ? (float)(kLptBins - 1) / mx : 0.f;
    auto bin_of = [&](int i) {
        int b = (int)(cost[i] * scale);
        b = b < 0 ? 0 : (b > kLptBins - 1 ? kLptBins - 1 : b);
        return kLptBins - 1 - b;  // bin 0 = most expensive
    };
    for (int i = threadIdx.x; i < nchunks; i += kLptThreads) atomicAdd(&hist[bin_of(i)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kLptBins; ++b) {
            int h = hist[b];
            hist[b] = acc;
            acc += h;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nchunks; i += kLptThreads)
        tmp[atomicAdd(&hist[bin_of(i)], 1)] = chunks[i];
    __syncthreads();
    for (int i = threadIdx.x; i < nchunks; i += kLptThreads) chunks[i] = tmp[i];
}

}  // namespace

void launch_chunk_order(int4* chunks, int nchunks, const int* targets, const int* cnt_p2p,
                        const int* cnt_m2p, float* cost, int4* tmp, cudaStream_t s)
{
    if (nchunks < 2) return;
    count_launch(2);
    k_chunk_cost<<<(nchunks + 7) / 8, 256, 0, s>>>(chunks, nchunks, targets, cnt_p2p, cnt_m2p,
                                                   cost);
    k_chunk_lpt<<<1, kLptThreads, 0, s>>>(chunks, nchunks, cost, tmp);
}

}  // namespace ucp
