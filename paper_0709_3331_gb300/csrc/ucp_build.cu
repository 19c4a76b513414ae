// ucp_build.cu -- TREE construction of Sec. 3 (arXiv 0709.3331) on the GPU:
// enclosing cube, Morton keys, stable radix sort, box topology as key
// prefixes in pre-order, and box moments bottom-up.
//
// Arithmetic that decides an integer (cube, cell coordinates, box centre) is
// written with explicit round-to-nearest intrinsics in the order of the
// definition, so that no multiply-add contraction changes a cell.
#include "ucp_internal.cuh"

#include <math.h>

namespace ucp {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread over a block of kScanThreads.
__device__ int block_excl_scan(int v, int* total)
{
    __shared__ int warp_sums[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v, lane);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        int si = warp_incl_scan(s, lane);
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == 31) *total = si;
    }
    __syncthreads();
    int r = warp_sums[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ part)
{
    int base = blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    __shared__ int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int* part, int nb, int* total)
{
    // one block: each thread scans a contiguous chunk of the partials
    int per = (nb + blockDim.x - 1) / blockDim.x;
    int b0 = threadIdx.x * per;
    int s = 0;
    for (int b = b0; b < b0 + per && b < nb; ++b) s += part[b];
    __shared__ int tot;
    int off = block_excl_scan(s, &tot);
    for (int b = b0; b < b0 + per && b < nb; ++b) {
        int v = part[b];
        part[b] = off;
        off += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void k_scan_apply(const int* __restrict__ in, int* __restrict__ out, int n,
                             const int* __restrict__ part)
{
    int base = blockIdx.x * kScanTile;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    __shared__ int tot;
    int off = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
}

// Target selection: the slots whose species is `species`, in slot order.  The
// count per tile and the write pass take the flag straight from the species.
__global__ void k_select_count(const int8_t* __restrict__ sp, int species, int n,
                               int* __restrict__ part)
{
    int base = blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        if (i < n) s += sp[i] == species;
    }
    __shared__ int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_select_write(const int8_t* __restrict__ sp, int species, int n,
                               const int* __restrict__ part, int* __restrict__ list)
{
    int base = blockIdx.x * kScanTile;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        v[k] = i < n && sp[i] == species;
        s += v[k];
    }
    __shared__ int tot;
    int off = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = base + threadIdx.x * kScanItems + k;
        if (v[k]) list[off++] = i;
    }
}

// ---------------------------------------------------------------- cube
// Ordered integer image of a finite double: comparing the images compares the
// values, so min/max run on the integer ALU instead of the (scarce) FP64 pipe.
// Partial min/max of cloud blockIdx.y over its segment (the whole array when
// cloud_start is NULL); block x of the cloud strides the segment.
__global__ void k_bbox_partial(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, int n, double* __restrict__ part,
                               const int* __restrict__ cloud_start)
{
    const int c = blockIdx.y;
    const int lo_i = cloud_start ? cloud_start[c] : 0, hi_i = cloud_start ? cloud_start[c + 1] : n;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int i = lo_i + blockIdx.x * blockDim.x + threadIdx.x; i < hi_i;
         i += gridDim.x * blockDim.x) {
        unsigned long long v[3] = {ord64(x[i]), ord64(y[i]), ord64(z[i])};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], v[a]);
            hi[a] = max(hi[a], v[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    __shared__ unsigned long long s[32][6];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            s[w][a] = lo[a];
            s[w][3 + a] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww)
            for (int a = 0; a < 3; ++a) {
                s[0][a] = min(s[0][a], s[ww][a]);
                s[0][3 + a] = max(s[0][3 + a], s[ww][3 + a]);
            }
        // an empty partial (more blocks than particles) keeps +/-inf
        double* pp = part + ((size_t)c * gridDim.x + blockIdx.x) * 6;
        for (int a = 0; a < 3; ++a) {
            pp[a] = s[0][a] == ~0ull ? INFINITY : unord64(s[0][a]);
            pp[3 + a] = s[0][3 + a] == 0ull ? -INFINITY : unord64(s[0][3 + a]);
        }
    }
}

// Sec. 3: the cube that encloses every particle.  Centre = (min + max) / 2 per
// axis; side = largest extent * (1 + 2^-20) so that the maximum falls inside;
// side 1 when all particles coincide.
__global__ void k_bbox_final(const double* __restrict__ part, int nblk, Cube* cubes)
{
    part += (size_t)blockIdx.x * nblk * 6;  // cloud blockIdx.x
    Cube* cube = cubes + blockIdx.x;
    // min and max taken on the ordered integer images, as in k_bbox_partial
    __shared__ unsigned long long s[256][6];
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], ord64(part[6 * b + a]));
            hi[a] = max(hi[a], ord64(part[6 * b + 3 + a]));
        }
    for (int a = 0; a < 3; ++a) {
        s[threadIdx.x][a] = lo[a];
        s[threadIdx.x][3 + a] = hi[a];
    }
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
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
        const double mn = unord64(s[0][a]), mx = unord64(s[0][3 + a]);
        cube->c[a] = __dmul_rn(__dadd_rn(mn, mx), 0.5);
        double e = __dsub_rn(mx, mn);
        if (e > ext) ext = e;
    }
    double L = ext > 0.0 ? __dmul_rn(ext, 1.0 + 0x1p-20) : 1.0;
    cube->L = L;
    for (int a = 0; a < 3; ++a) cube->lo[a] = __dsub_rn(cube->c[a], __dmul_rn(L, 0.5));
    cube->kscale = __ddiv_rn(2097152.0, L);
}

// ---------------------------------------------------------------- keys
__device__ __forceinline__ unsigned long long spread3(unsigned int v)
{
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// cell coordinate k = floor((x - lo) * (2^21 / L)), clamped to [0, 2^21 - 1].
// Truncation toward zero equals floor wherever the clamp keeps the value (it
// differs only below 0, which clamps to 0 either way), and the saturating
// conversion keeps values past the int range above the upper clamp: three FP64
// operations per axis, the clamps on the integer ALU.
__device__ __forceinline__ unsigned int cell_coord(double x, double lo, double kscale)
{
    const int k = __double2int_rz(__dmul_rn(__dsub_rn(x, lo), kscale));
    return (unsigned int)min(max(k, 0), 2097151);
}

__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, int n, const Cube* __restrict__ cubes,
                       const unsigned char* __restrict__ cloud,
                       unsigned long long* __restrict__ key, unsigned int* __restrict__ val)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Cube* cube = cubes + (cloud ? cloud[i] : 0);
    double ks = cube->kscale;
    unsigned int kx = cell_coord(x[i], cube->lo[0], ks);
    unsigned int ky = cell_coord(y[i], cube->lo[1], ks);
    unsigned int kz = cell_coord(z[i], cube->lo[2], ks);
    key[i] = spread3(kx) | (spread3(ky) << 1) | (spread3(kz) << 2);
    val[i] = (unsigned int)i;
}

// ---------------------------------------------------------------- sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortChunks = 8;                              // 32-key chunks per warp
constexpr int kSortTile = kSortThreads * kSortChunks;       // 2048 keys per block
constexpr int kRadix = 256;
constexpr int kSortSpinLimit = 1 << 20;  // polls of a predecessor's word before giving up
constexpr int kLook = 8;                  // predecessors read per look-back round trip

// Digit histograms of all eight passes in one read of the keys.
__global__ void __launch_bounds__(kSortThreads)
k_sort_hist_all(const unsigned long long* __restrict__ key, int n, unsigned int* __restrict__ ghist)
{
    __shared__ unsigned int h[8][kRadix];
    for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int i = blockIdx.x * kSortThreads + threadIdx.x; i < n; i += gridDim.x * kSortThreads) {
        unsigned long long k = key[i];
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(unsigned int)(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) {
        unsigned int v = (&h[0][0])[i];
        if (v) atomicAdd(&ghist[i], v);
    }
}

// goff[p][d] = number of keys whose pass-p digit is below d.
// Also advances the sort's tag: every build's published words carry a tag 16
// above the previous build's, kept on the device so that a captured graph
// replays with fresh tags (every word of a pass region is rewritten each build,
// so a stale word always carries an older tag, also across 30-bit wrap-around).
__global__ void __launch_bounds__(kRadix) k_sort_offsets(const unsigned int* __restrict__ ghist,
                                                         unsigned int* __restrict__ goff,
                                                         unsigned int* __restrict__ epoch)
{
    __shared__ int tot;
    if (threadIdx.x == 0) *epoch = (*epoch + 16u) & 0x3fffffffu;
    for (int p = 0; p < 8; ++p) {
        int v = (int)ghist[p * kRadix + threadIdx.x];
        goff[p * kRadix + threadIdx.x] = (unsigned int)block_excl_scan(v, &tot);
    }
}

// One stable LSD pass in a single kernel (decoupled look-back).  A block takes
// the next tile from a counter, ranks its keys stably (each warp owns a
// contiguous quarter-tile and ranks it chunk by chunk with match_any), and
// publishes its per-digit count; the digit offset of the tile is the sum of
// the counts of all earlier tiles, read back through their published words
// {epoch, flag (1 = count of the tile, 2 = inclusive prefix), value}.  A block
// waits only on tiles taken before its own, whose blocks are running, and
// every wait is bounded: past spin_limit polls it raises *err, keeps its keys
// where they are and leaves (the host reports UCP_ETIMEOUT).
__global__ void __launch_bounds__(kSortThreads)
k_onesweep(const unsigned long long* __restrict__ kin, const unsigned int* __restrict__ vin,
           unsigned long long* __restrict__ kout, unsigned int* __restrict__ vout, int n,
           int shift, const unsigned int* __restrict__ goff, unsigned long long* status,
           int* tile_ctr, const unsigned int* __restrict__ epoch_dev, unsigned int pass, int* err,
           int spin_limit, const unsigned char* __restrict__ digit_of_val)
{
    const unsigned int epoch = (*epoch_dev + pass) & 0x3fffffffu;
    __shared__ int cnt[kSortWarps][kRadix];
    __shared__ int s_tile, s_fail;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_ctr, 1);
        s_fail = 0;
    }
    for (int d = lane; d < kRadix; d += 32) cnt[w][d] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int base = tile * kSortTile + w * (kSortTile / kSortWarps);
    unsigned long long kk[kSortChunks];
    unsigned int vv[kSortChunks];
    int dig[kSortChunks], rank[kSortChunks];
    const unsigned int lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        int i = base + c * 32 + lane;
        bool ok = i < n;
        kk[c] = ok ? kin[i] : 0ull;
        vv[c] = ok ? vin[i] : 0u;
        // digit: 8 key bits, or (cloud pass) the cloud of the element's previous slot
        int d = ok ? (digit_of_val ? (int)digit_of_val[vv[c]] : (int)((kk[c] >> shift) & 0xffu))
                   : kRadix + lane;  // invalid lanes unique
        dig[c] = d;
        unsigned int peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int before = 0;
        if (ok && lane == leader) {
            before = cnt[w][d];
            cnt[w][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[c] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // kSortThreads == kRadix
        int total = 0;
        for (int ww = 0; ww < kSortWarps; ++ww) {
            int t = cnt[ww][d];
            cnt[ww][d] = total;
            total += t;
        }
        const unsigned long long tag = (unsigned long long)epoch << 34;
        unsigned long long* mine = status + (size_t)tile * kRadix + d;
        unsigned int prefix = 0;
        if (tile > 0) {
            atomicExch(mine, tag | (1ull << 32) | (unsigned int)total);
            // kLook predecessors' words per round trip (independent loads), taken in
            // order j, j - 1, ... up to the first inclusive prefix or the first word
            // not yet published, which is polled again
            int j = tile - 1, spins = 0;
            bool done = false;
            while (!done) {
                unsigned long long v[kLook];
#pragma unroll
                for (int u = 0; u < kLook; ++u)
                    v[u] = j - u >= 0 ? __ldcv(status + (size_t)(j - u) * kRadix + d) : 0ull;
                int used = 0;
                bool blocked = false;
#pragma unroll
                for (int u = 0; u < kLook; ++u) {
                    if (done || blocked || j - u < 0) continue;
                    const unsigned int flag = (unsigned int)(v[u] >> 32) & 3u;
                    if ((v[u] >> 34) != (unsigned long long)epoch || flag == 0u) {
                        blocked = true;
                        continue;
                    }
                    prefix += (unsigned int)v[u];
                    ++used;
                    if (flag == 2u) done = true;
                }
                j -= used;
                if (done || j < 0) break;  // (tile 0 publishes an inclusive prefix)
                if (blocked) {
                    if (++spins > spin_limit) {
                        atomicOr(err, 1);
                        s_fail = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        atomicExch(mine, tag | (2ull << 32) | (prefix + (unsigned int)total));
        const int off = (int)(goff[d] + prefix);
        for (int ww = 0; ww < kSortWarps; ++ww) cnt[ww][d] += off;
    }
    __syncthreads();
    const bool fail = s_fail != 0;
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        int i = base + c * 32 + lane;
        if (i < n) {
            int p = fail ? i : cnt[w][dig[c]] + rank[c];
            kout[p] = kk[c];
            vout[p] = vv[c];
        }
    }
}

// Equal keys must come out ordered by caller index (ties by particle index):
// the run starting at i is insertion-sorted by ids[perm[.]].  Runs are rare and
// short except when particles coincide (depth-21 boxes).
__global__ void k_tiefix(const unsigned long long* __restrict__ key, unsigned int* __restrict__ perm,
                         const unsigned int* __restrict__ ids, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    unsigned long long k = key[i];
    if (key[i + 1] != k || (i > 0 && key[i - 1] == k)) return;
    int e = i + 1;
    while (e < n && key[e] == k) ++e;
    for (int a = i + 1; a < e; ++a) {
        unsigned int pv = perm[a];
        unsigned int idv = ids[pv];
        int b = a - 1;
        while (b >= i && ids[perm[b]] > idv) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = pv;
    }
}

// ---------------------------------------------------------------- topology
__device__ __forceinline__ unsigned long long prefix_at(unsigned long long k, int d)
{
    return d == 0 ? 0ull : (k >> (3 * (kMaxDepth - d)));
}

// Boxes never span two clouds: every cloud occupies a fixed segment
// [seg_lo, seg_hi) of the key-sorted order (its own root, its own cube).

// first j > i in the segment whose depth-d prefix differs from key[i]'s (or seg_hi)
__device__ int box_end(const unsigned long long* __restrict__ K, int seg_hi, int i, int d)
{
    if (d == 0) return seg_hi;
    unsigned long long p = prefix_at(K[i], d);
    int lo = i, step = 1, hi = i + 1;
    while (hi < seg_hi && prefix_at(K[hi], d) == p) {
        lo = hi;
        step <<= 1;
        hi = i + step;
    }
    if (hi > seg_hi) hi = seg_hi;
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if (prefix_at(K[mid], d) == p) lo = mid;
        else hi = mid;
    }
    return hi;
}

// first j <= i in the segment whose depth-d prefix equals key[i]'s
__device__ int box_begin(const unsigned long long* __restrict__ K, int seg_lo, int i, int d)
{
    if (d == 0) return seg_lo;
    unsigned long long p = prefix_at(K[i], d);
    int hi = i, step = 1, lo = i - 1;
    while (lo >= seg_lo && prefix_at(K[lo], d) == p) {
        hi = lo;
        step <<= 1;
        lo = i - step;
    }
    if (lo < seg_lo - 1) lo = seg_lo - 1;
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if (prefix_at(K[mid], d) == p) hi = mid;
        else lo = mid;
    }
    return hi;
}

// depth of the first box that starts at sorted position i (22 = none)
__device__ __forceinline__ int first_depth(const unsigned long long* __restrict__ K, int seg_lo,
                                           int i)
{
    if (i == seg_lo) return 0;
    unsigned long long x = K[i] ^ K[i - 1];
    if (x == 0ull) return kMaxDepth + 1;
    return (__clzll((long long)x) - 1) / 3 + 1;
}

__device__ __forceinline__ void segment_of(const Tree& t, int n, int i, int& lo, int& hi)
{
    if (t.cloud) {
        const int c = t.cloud[i];
        lo = t.cloud_start[c];
        hi = t.cloud_start[c + 1];
    } else {
        lo = 0;
        hi = n;
    }
}

// Every box is a key prefix; the boxes that start at sorted position i are
// those of depth >= first_depth(i) down to the first leaf.  A box exists iff
// its parent holds more than leaf_cap particles.  Emitting boxes in order of
// (start position, depth) gives pre-order with children in octant order.
__global__ void k_topo_count(const unsigned long long* __restrict__ K, int n, int leaf_cap,
                             int* __restrict__ cnt, Tree t)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo, hi;
    segment_of(t, n, i, lo, hi);
    int d0 = first_depth(K, lo, i);
    int c = 0;
    if (d0 <= kMaxDepth) {
        bool ok = true;
        if (d0 > 0) {
            int pb = box_begin(K, lo, i, d0 - 1), pe = box_end(K, hi, i, d0 - 1);
            ok = pe - pb > leaf_cap;
        }
        if (ok)
            for (int d = d0; d <= kMaxDepth; ++d) {
                int e = box_end(K, hi, i, d);
                ++c;
                if (e - i <= leaf_cap || d == kMaxDepth) break;
            }
    }
    cnt[i] = c;
}

// ---- the same counts by a window of sorted positions (leaf_cap <= kTopoWin).
// fd[j] = first_depth(j): the box of depth d that holds position i ends at the
// first j > i with fd[j] <= d and starts at the last j <= i with fd[j] <= d.  It
// holds at most leaf_cap particles iff those two lie within leaf_cap of each
// other, so the depth of the leaf that holds i is
//   min over m = 0 .. leaf_cap - 1 of max(min fd[i - m .. i], min fd[i + 1 .. i + leaf_cap - m])
// (capped at kMaxDepth): a fixed window of shared memory instead of searches.
// Outside [0, n) and at every segment start fd is 0, which closes every box.
constexpr int kTopoThreads = 256;
constexpr int kTopoWin = 32;

__device__ __forceinline__ int fd_at(const unsigned long long* __restrict__ K, const Tree& t,
                                     int n, int j)
{
    if (j <= 0 || j >= n) return 0;
    int lo, hi;
    segment_of(t, n, j, lo, hi);
    return first_depth(K, lo, j);
}

// fd over [base - kTopoWin, base + kTopoThreads + kTopoWin) into smem
__device__ __forceinline__ void load_fd_window(const unsigned long long* __restrict__ K,
                                               const Tree& t, int n, int base,
                                               unsigned char* fd)
{
    for (int k = threadIdx.x; k < kTopoThreads + 2 * kTopoWin; k += kTopoThreads)
        fd[k] = (unsigned char)fd_at(K, t, n, base - kTopoWin + k);
}

// depth of the leaf that holds the position in slot li (see above); the
// backward running minima stay in registers (fully unrolled over the window)
__device__ __forceinline__ int leaf_depth_win(const unsigned char* fd, int li, int w)
{
    int bmin[kTopoWin];
    int bm = 255;
#pragma unroll
    for (int m = 0; m < kTopoWin; ++m) {
        if (m < w) bm = min(bm, (int)fd[li - m]);
        bmin[m] = bm;
    }
    int fm = 255, best = 255;
#pragma unroll
    for (int m = kTopoWin - 1; m >= 0; --m) {
        if (m < w) {
            fm = min(fm, (int)fd[li + (w - m)]);
            best = min(best, max(bmin[m], fm));
        }
    }
    return min(best, kMaxDepth);
}

__global__ void __launch_bounds__(kTopoThreads)
k_topo_count_win(const unsigned long long* __restrict__ K, int n, int leaf_cap,
                 int* __restrict__ cnt, Tree t)
{
    __shared__ unsigned char fd[kTopoThreads + 2 * kTopoWin];
    const int base = blockIdx.x * kTopoThreads;
    load_fd_window(K, t, n, base, fd);
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i >= n) return;
    const int li = threadIdx.x + kTopoWin;
    const int d0 = fd[li];
    int c = 0;
    if (d0 <= kMaxDepth) {
        const int lv = leaf_depth_win(fd, li, leaf_cap);
        if (lv >= d0) c = lv - d0 + 1;
    }
    cnt[i] = c;
}

// atomicAdd(ctr, 1) for every calling lane, one atomic per distinct counter in
// the warp (the lanes that add to the same counter take consecutive slots)
__device__ __forceinline__ int warp_inc(int* ctr)
{
    const unsigned int active = __activemask();
    const unsigned int peers = __match_any_sync(active, (unsigned long long)ctr);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(ctr, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

template <bool kWin>
__global__ void __launch_bounds__(kTopoThreads)
k_topo_emit(const unsigned long long* __restrict__ K, int n, int leaf_cap,
            const int* __restrict__ cnt, const int* __restrict__ off, Tree t)
{
    // with kWin the leaf's end comes from the window of first depths (a leaf
    // holds at most leaf_cap <= kTopoWin positions unless it is a depth-cap box)
    __shared__ unsigned char fd[kWin ? kTopoThreads + 2 * kTopoWin : 1];
    if (kWin) {
        load_fd_window(K, t, n, blockIdx.x * kTopoThreads, fd);
        __syncthreads();
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cnt[i];
    // the capacity bounds the box count of sorted keys; clamp in case it ever did not
    int nn = min(*t.nnodes, t.cap);
    if (i == 0 && *t.nnodes > t.cap) *t.nnodes = t.cap;
    if (c == 0) return;
    int lo, hi;
    segment_of(t, n, i, lo, hi);
    int d0 = first_depth(K, lo, i);
    int node = off[i];
    int parent = -1;
    if (d0 > 0) {
        int pb = box_begin(K, lo, i, d0 - 1);
        parent = off[pb] + (d0 - 1 - first_depth(K, lo, pb));
    }
    int dmax = 0;
    for (int j = 0; j < c; ++j) {
        int d = d0 + j;
        // the boxes above the last one at this position hold more than leaf_cap
        // particles (the count stops at the first that does not): twigs, whose end
        // and skip index are their last child's, filled in by the moments' bottom-up
        // sweep; only the last box's end is looked up here
        int e = -1, nx = -1;
        bool leaf = false;
        if (j == c - 1) {
            if (kWin) {
                // the leaf: its end within the window, else (a bigger depth-cap box) search
                const int li = threadIdx.x + kTopoWin;
                for (int m = 1; m <= leaf_cap && e < 0; ++m)
                    if (fd[li + m] <= d) e = i + m;
            }
            if (e < 0) e = box_end(K, hi, i, d);
            leaf = (e - i <= leaf_cap) || d == kMaxDepth;
            nx = e < n ? off[e] : nn;
        }
        if (node >= t.cap) break;  // cannot happen: the capacity bounds the box count
        unsigned long long pre = prefix_at(K[i], d);
        t.info[node] = make_int4(i, e, nx, parent);
        t.depth_leaf[node] = d | (leaf ? 256 : 0);
        t.cell[node] = pre;
        if (parent >= 0) t.child8[(size_t)parent * 8 + (int)(pre & 7ull)] = node;
        int* ctr = &t.count[leaf ? kMaxDepth + 1 : d];
        const int slot = warp_inc(ctr);
        if (leaf) t.leaf_list[slot] = node;
        else t.twig_list[t.twig_off[d] + slot] = node;
        parent = node;
        ++node;
        dmax = d;
    }
    atomicMax(t.maxdepth, dmax);
}

// ---------------------------------------------------------------- moments
__device__ __forceinline__ unsigned int compact3(unsigned long long x)
{
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x | (x >> 4)) & 0x100f00f00f00f00full;
    x = (x | (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x | (x >> 16)) & 0x001f00000000ffffull;
    x = (x | (x >> 32)) & 0x1fffffull;
    return (unsigned int)x;
}

// cube of the cloud that owns the box starting at sorted position i
__device__ __forceinline__ Cube cube_of(const Cube* __restrict__ cubes, const Tree& t, int i)
{
    return cubes[t.cloud ? t.cloud[i] : 0];
}

// geometric box centre: lo + (cell + 1/2) * side, side = L 2^-depth
__device__ __forceinline__ void box_centre(const Cube& cb, unsigned long long cell, int d,
                                           double ctr[3], double* side)
{
    double s = ldexp(cb.L, -d);
    *side = s;
    unsigned int ic[3] = {compact3(cell), compact3(cell >> 1), compact3(cell >> 2)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double lo = __dsub_rn(cb.c[a], __dmul_rn(cb.L, 0.5));
        ctr[a] = __dadd_rn(lo, __dmul_rn(__dadd_rn((double)ic[a], 0.5), s));
    }
}

// Moments of one box from sums about its geometric centre z:
//   a = {S0, M, sum|q|y (3), sum q y (3), sum q y y^T (6)},  y = x - z.
// The expansion centre is the |q|-weighted centroid c = z + e, e = sum|q|y / S0
// (z when S0 = 0); shifting to c: D = sum q y - M e,
// Q = sum q y y^T - (sum q y) e^T - e (sum q y)^T + M e e^T.  delta = |e|.
__device__ __forceinline__ void finish_box(const double* a, const double z[3],
                                           double* __restrict__ m)
{
    double S0 = a[0], M = a[1];
    double e[3];
    const double inv = S0 > 0.0 ? 1.0 / S0 : 0.0;
    for (int k = 0; k < 3; ++k) e[k] = a[2 + k] * inv;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = a[5 + k];
    m[MC + 0] = z[0] + e[0];
    m[MC + 1] = z[1] + e[1];
    m[MC + 2] = z[2] + e[2];
    m[MM] = M;
    for (int k = 0; k < 3; ++k) m[MD + k] = d[k] - M * e[k];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k)
        m[MQ + k] = a[8 + k] - d[ia[k]] * e[ib[k]] - e[ia[k]] * d[ib[k]] + M * e[ia[k]] * e[ib[k]];
    m[MS0] = S0;
    // delta = |c - z| rounded like the definition: c is stored first, then differenced
    double ex = __dsub_rn(m[MC + 0], z[0]);
    double ey = __dsub_rn(m[MC + 1], z[1]);
    double ez = __dsub_rn(m[MC + 2], z[2]);
    m[MDELTA] = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                     __dmul_rn(ez, ez)));
}

__global__ void k_clear_children(Tree t)
{
    int total = *t.nnodes * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        t.child8[i] = -1;
}

// Moments of twig p (depth d) from its eight child slots in octant order, each
// child's moments shifted to the twig's geometric centre.  The children were
// written by other threads of the same launch: their records are read through
// L2 (__ldcg) after the fence of the bottom-up sweep.
__device__ void twig_combine_f64(const Cube* __restrict__ cube, const Tree& t, int p, int d)
{
    const Cube cb = cube_of(cube, t, t.info[p].x);
    double zp[3], ps;
    box_centre(cb, t.cell[p], d, zp, &ps);
    double a[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) a[k] = 0.0;
#pragma unroll 1
    for (int o = 0; o < 8; ++o) {
        const int ch = t.child8[(size_t)p * 8 + o];
        if (ch < 0) continue;
        const double* cm = t.mom + (size_t)ch * kMom;
        double S0k = __ldcg(cm + MS0), Mk = __ldcg(cm + MM);
        double e[3], dk[3], qk[6];
        for (int k = 0; k < 3; ++k) {
            e[k] = __ldcg(cm + MC + k) - zp[k];
            dk[k] = __ldcg(cm + MD + k);
        }
        for (int k = 0; k < 6; ++k) qk[k] = __ldcg(cm + MQ + k);
        a[0] += S0k;
        a[1] += Mk;
        for (int k = 0; k < 3; ++k) {
            a[2 + k] += S0k * e[k];
            a[5 + k] += dk[k] + Mk * e[k];
        }
        // Q_k + D_k e^T + e D_k^T + M_k e e^T
        double me0 = Mk * e[0], me1 = Mk * e[1], me2 = Mk * e[2];
        a[8] += qk[0] + (2.0 * dk[0] + me0) * e[0];
        a[9] += qk[1] + dk[0] * e[1] + (dk[1] + me1) * e[0];
        a[10] += qk[2] + dk[0] * e[2] + (dk[2] + me2) * e[0];
        a[11] += qk[3] + (2.0 * dk[1] + me1) * e[1];
        a[12] += qk[4] + dk[1] * e[2] + (dk[2] + me2) * e[1];
        a[13] += qk[5] + (2.0 * dk[2] + me2) * e[2];
    }
    double rec[kMom];
    finish_box(a, zp, rec);
    double* pm = t.mom + (size_t)p * kMom;
#pragma unroll
    for (int k = 0; k < kMom; ++k) pm[k] = rec[k];
}

constexpr int kMomThreads = 64;  // threads per block of the leaf kernels

// atomicAdd with acquire-release semantics at device scope: the caller's
// earlier writes are visible to whoever reads the counter after it (release),
// and the writes released by every earlier increment of the counter are
// visible to the caller after it (acquire: the increments form one release
// sequence).  One ordered atomic in place of a fence on either side.
__device__ __forceinline__ int atomic_add_acq_rel(int* ctr, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
                 : "=r"(old) : "l"(ctr), "r"(v) : "memory");
    return old;
}

// Bottom-up sweep from a finished box: each box counts its finished children
// (t.arrive, zeroed before the launch); the thread that finishes the last child
// combines the parent and carries on upwards.  No thread waits for another, and
// every twig is combined once, from all its children, whichever thread does it.
template <class Combine>
__device__ __forceinline__ void sweep_up(const Tree& t, int node, Combine combine)
{
    int p = t.info[node].w;
    while (p >= 0) {
        int nch = 0, last = -1;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ch = t.child8[(size_t)p * 8 + o];
            nch += ch >= 0;
            if (ch >= 0) last = ch;
        }
        // this box's records are published with its arrival; the last arrival
        // sees every sibling's
        if (atomic_add_acq_rel(&t.arrive[p], 1) + 1 < nch) return;
        // a twig ends where its last child (in octant order, so last in pre-order)
        // ends, and skips to where that child skips
        const int4 lc = __ldcg(&t.info[last]);
        int* ip = reinterpret_cast<int*>(&t.info[p]);
        ip[1] = lc.y;
        ip[2] = lc.z;
        combine(p, t.depth_leaf[p] & 255);
        p = t.info[p].w;
    }
}

// Moments of every leaf from its particles, one thread per leaf, summed about
// the leaf's geometric centre in key order.
__global__ void __launch_bounds__(kMomThreads)
k_moments_leaves(const double* __restrict__ x, const double* __restrict__ y,
                 const double* __restrict__ z, const int8_t* __restrict__ sp,
                 const double* __restrict__ qsp, const Cube* __restrict__ cube, Tree t,
                 float4* __restrict__ src32, int want_f32)
{
    const int nl = t.count[kMaxDepth + 1];
    const double q0 = qsp[0], q1 = qsp[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
        const int node = t.leaf_list[i];
        const int dl = t.depth_leaf[node];
        const int4 inf = t.info[node];
        const Cube cb = cube_of(cube, t, inf.x);
        double zc[3], side;
        box_centre(cb, t.cell[node], dl & 255, zc, &side);
        double a[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) a[k] = 0.0;
        for (int j = inf.x; j < inf.y; ++j) {
            double qj = sp[j] ? q1 : q0;
            double aq = fabs(qj);
            double yv[3] = {x[j] - zc[0], y[j] - zc[1], z[j] - zc[2]};
            a[0] += aq;
            a[1] += qj;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a[2 + k] += aq * yv[k];
                a[5 + k] += qj * yv[k];
            }
            double qy0 = qj * yv[0], qy1 = qj * yv[1];
            a[8] += qy0 * yv[0];
            a[9] += qy0 * yv[1];
            a[10] += qy0 * yv[2];
            a[11] += qy1 * yv[1];
            a[12] += qy1 * yv[2];
            a[13] += qj * yv[2] * yv[2];
        }
        double rec[kMom];
        finish_box(a, zc, rec);
        double* m = t.mom + (size_t)node * kMom;
#pragma unroll
        for (int k = 0; k < kMom; ++k) m[k] = rec[k];
        if (want_f32) {
            // paired layout: src32[2p] = {nx_2p, nx_2p+1, ny_2p, ny_2p+1},
            // src32[2p+1] = {nz_2p, nz_2p+1, q_2p, q_2p+1}, n = c_leaf - x
            float* f = reinterpret_cast<float*>(src32);
            for (int j = inf.x; j < inf.y; ++j) {
                double qj = sp[j] ? q1 : q0;
                size_t b = (size_t)(j >> 1) * 8 + (j & 1);
                f[b] = (float)(rec[MC] - x[j]);
                f[b + 2] = (float)(rec[MC + 1] - y[j]);
                f[b + 4] = (float)(rec[MC + 2] - z[j]);
                f[b + 6] = (float)qj;
            }
        }
        sweep_up(t, node, [&](int p, int d) { twig_combine_f64(cube, t, p, d); });
    }
}

// ---- FP32 moments (FP32C contexts).  Offsets from a box's geometric centre z
// are at most one box side, so they are formed in FP64 once and summed in FP32;
// the expansion centre is c = z + e exactly as stored (FP64), and D, Q are taken
// about that same point.  Compact per-box record mom32 = {e xyz, S0, M, D xyz,
// Q xx xy xz yy yz zz, 0, 0} feeds the twig combine.
__device__ __forceinline__ void finish_box_f32(const float* a, const double z[3], float* m32,
                                               double* __restrict__ m64)
{
    float S0 = a[0], M = a[1];
    float inv = S0 > 0.f ? 1.f / S0 : 0.f;
    float e[3] = {a[2] * inv, a[3] * inv, a[4] * inv};
    float d[3];
    for (int k = 0; k < 3; ++k) d[k] = fmaf(-M, e[k], a[5 + k]);
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    float q[6];
    for (int k = 0; k < 6; ++k)
        q[k] = a[8 + k] - a[5 + ia[k]] * e[ib[k]] - e[ia[k]] * a[5 + ib[k]] +
               M * e[ia[k]] * e[ib[k]];
    m32[0] = e[0];
    m32[1] = e[1];
    m32[2] = e[2];
    m32[3] = S0;
    m32[4] = M;
    for (int k = 0; k < 3; ++k) m32[5 + k] = d[k];
    for (int k = 0; k < 6; ++k) m32[8 + k] = q[k];
    m32[14] = 0.f;
    m32[15] = 0.f;
    for (int k = 0; k < 3; ++k) m64[MC + k] = z[k] + (double)e[k];
    m64[MM] = M;
    for (int k = 0; k < 3; ++k) m64[MD + k] = d[k];
    for (int k = 0; k < 6; ++k) m64[MQ + k] = q[k];
    m64[MS0] = S0;
    m64[MDELTA] = sqrtf(fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2])));
}

// Child slot o of twig p shifted to the twig's centre (zeros for an empty slot).
// The child's expansion centre lies at its own geometric centre plus its FP32
// offset e_child (mom32), and its geometric centre at the twig's plus q = side/4
// along each axis, signed by the octant bit (x bit 0, y bit 1, z bit 2): the shift
// is q +/- e_child, formed in FP32 without touching the FP64 unit.
__device__ __forceinline__ void twig_child_f32(const Tree& t, int p, int o, float q, float* a)
{
#pragma unroll
    for (int k = 0; k < 14; ++k) a[k] = 0.f;
    const int ch = t.child8[(size_t)p * 8 + o];
    if (ch < 0) return;
    const float4* r32 = reinterpret_cast<const float4*>(t.mom32 + (size_t)ch * 16);
    const float4 R0 = __ldcg(r32), R1 = __ldcg(r32 + 1), R2 = __ldcg(r32 + 2),
                 R3 = __ldcg(r32 + 3);
    const float S0k = R0.w, Mk = R1.x;
    const float dk[3] = {R1.y, R1.z, R1.w};
    const float qk[6] = {R2.x, R2.y, R2.z, R2.w, R3.x, R3.y};
    const float ec[3] = {R0.x, R0.y, R0.z};
    float e[3];
    for (int k = 0; k < 3; ++k) e[k] = ((o >> k) & 1 ? q : -q) + ec[k];
    a[0] = S0k;
    a[1] = Mk;
    for (int k = 0; k < 3; ++k) {
        a[2 + k] = S0k * e[k];
        a[5 + k] = fmaf(Mk, e[k], dk[k]);
    }
    float me0 = Mk * e[0], me1 = Mk * e[1], me2 = Mk * e[2];
    a[8] = qk[0] + (2.f * dk[0] + me0) * e[0];
    a[9] = qk[1] + dk[0] * e[1] + (dk[1] + me1) * e[0];
    a[10] = qk[2] + dk[0] * e[2] + (dk[2] + me2) * e[0];
    a[11] = qk[3] + (2.f * dk[1] + me1) * e[1];
    a[12] = qk[4] + dk[1] * e[2] + (dk[2] + me2) * e[1];
    a[13] = qk[5] + (2.f * dk[2] + me2) * e[2];
}

// FP32 moments of twig p (depth d) from its eight shifted child slots, summed as
// ((s0 + s4) + (s2 + s6)) + ((s1 + s5) + (s3 + s7)): the order of an xor
// butterfly over the slots.
__device__ void twig_combine_f32(const Cube* __restrict__ cube, const Tree& t, int p, int d)
{
    const Cube cb = cube_of(cube, t, t.info[p].x);
    double zp[3], ps;
    box_centre(cb, t.cell[p], d, zp, &ps);
    const float q = (float)(0.25 * ps);
    float u[14], v[14], w[14];
    const int order[4][2] = {{0, 4}, {2, 6}, {1, 5}, {3, 7}};
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        float b0[14], b1[14];
        twig_child_f32(t, p, order[g][0], q, b0);
        twig_child_f32(t, p, order[g][1], q, b1);
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float s = b0[k] + b1[k];
            if (g == 0) u[k] = s;
            else if (g == 1) u[k] = u[k] + s;
            else if (g == 2) v[k] = s;
            else v[k] = v[k] + s;
        }
    }
#pragma unroll
    for (int k = 0; k < 14; ++k) w[k] = u[k] + v[k];
    float m32[16];
    finish_box_f32(w, zp, m32, t.mom + (size_t)p * kMom);
    float4* w32 = reinterpret_cast<float4*>(t.mom32 + (size_t)p * 16);
    for (int k = 0; k < 4; ++k)
        w32[k] = make_float4(m32[4 * k], m32[4 * k + 1], m32[4 * k + 2], m32[4 * k + 3]);
}

// Leaves, one thread per leaf (full lanes for the FP64 offsets), then the
// bottom-up sweep over the twigs (sweep_up).
__global__ void __launch_bounds__(kMomThreads)
k_moments_leaves_f32(const double* __restrict__ x, const double* __restrict__ y,
                     const double* __restrict__ z, const int8_t* __restrict__ sp,
                     const double* __restrict__ qsp, const Cube* __restrict__ cube, Tree t,
                     float4* __restrict__ src32)
{
    const int nl = t.count[kMaxDepth + 1];
    const float q0 = (float)qsp[0], q1 = (float)qsp[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
        const int node = t.leaf_list[i];
        const int dl = t.depth_leaf[node];
        const int4 inf = t.info[node];
        const Cube cb = cube_of(cube, t, inf.x);
        double zc[3], side;
        box_centre(cb, t.cell[node], dl & 255, zc, &side);
        float a[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) a[k] = 0.f;
#pragma unroll 4
        for (int j = inf.x; j < inf.y; ++j) {
            float qj = sp[j] ? q1 : q0;
            float aq = fabsf(qj);
            float yv[3] = {(float)(x[j] - zc[0]), (float)(y[j] - zc[1]), (float)(z[j] - zc[2])};
            a[0] += aq;
            a[1] += qj;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a[2 + k] = fmaf(aq, yv[k], a[2 + k]);
                a[5 + k] = fmaf(qj, yv[k], a[5 + k]);
            }
            float qy0 = qj * yv[0], qy1 = qj * yv[1];
            a[8] = fmaf(qy0, yv[0], a[8]);
            a[9] = fmaf(qy0, yv[1], a[9]);
            a[10] = fmaf(qy0, yv[2], a[10]);
            a[11] = fmaf(qy1, yv[1], a[11]);
            a[12] = fmaf(qy1, yv[2], a[12]);
            a[13] = fmaf(qj * yv[2], yv[2], a[13]);
        }
        float m32[16];
        double* m = t.mom + (size_t)node * kMom;
        finish_box_f32(a, zc, m32, m);
        float4* r32 = reinterpret_cast<float4*>(t.mom32 + (size_t)node * 16);
        for (int k = 0; k < 4; ++k)
            r32[k] = make_float4(m32[4 * k], m32[4 * k + 1], m32[4 * k + 2], m32[4 * k + 3]);
        // paired sources: src32[2p] = {nx_2p, nx_2p+1, ny_2p, ny_2p+1},
        // src32[2p+1] = {nz_2p, nz_2p+1, q_2p, q_2p+1}, n = c_leaf - x
        const double cx = m[MC], cy = m[MC + 1], cz = m[MC + 2];
        float* f = reinterpret_cast<float*>(src32);
        for (int j = inf.x; j < inf.y; ++j) {
            size_t b = (size_t)(j >> 1) * 8 + (j & 1);
            f[b] = (float)(cx - x[j]);
            f[b + 2] = (float)(cy - y[j]);
            f[b + 4] = (float)(cz - z[j]);
            f[b + 6] = sp[j] ? q1 : q0;
        }
        sweep_up(t, node, [&](int p, int d) { twig_combine_f32(cube, t, p, d); });
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers
size_t scan_partials_words(int n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

void launch_scan(const int* in, int* out, int n, int* partials, int* total, cudaStream_t s)
{
    count_launch(3);
    int nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, partials);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, nb, total);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, partials);
}

void launch_select(const int8_t* sp, int species, int n, int* list, int* partials, int* count,
                   cudaStream_t s)
{
    count_launch(3);
    int nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    k_select_count<<<nb, kScanThreads, 0, s>>>(sp, species, n, partials);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, nb, count);
    k_select_write<<<nb, kScanThreads, 0, s>>>(sp, species, n, partials, list);
}

void launch_bbox(const double* x, const double* y, const double* z, int n, double* partials,
                 int nblk, Cube* cubes, const int* cloud_start, int n_clouds, cudaStream_t s)
{
    count_launch(2);
    k_bbox_partial<<<dim3(nblk, n_clouds), 256, 0, s>>>(x, y, z, n, partials, cloud_start);
    k_bbox_final<<<n_clouds, 256, 0, s>>>(partials, nblk, cubes);
}

void launch_keys(const double* x, const double* y, const double* z, int n, const Cube* cubes,
                 const unsigned char* cloud, unsigned long long* key, unsigned int* val,
                 cudaStream_t s)
{
    count_launch(1);
    k_keys<<<(n + 255) / 256, 256, 0, s>>>(x, y, z, n, cubes, cloud, key, val);
}

size_t sort_test_words() { return 4 * (size_t)kSortTile; }

size_t sort_status_words(int n)
{
    int nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)9 * kRadix * (size_t)(nb > 0 ? nb : 1);
}

int launch_sort(unsigned long long* key[2], unsigned int* val[2], int n, SortScratch sc,
                const unsigned int* ids_in, const unsigned char* cloud,
                const int* cloud_start, int n_clouds, cudaStream_t s)
{
    count_launch(11 + (n_clouds > 1 ? 1 : 0));
    const int nb = (n + kSortTile - 1) / kSortTile;
    cudaMemsetAsync(sc.ghist, 0, sizeof(unsigned int) * (8 * kRadix + 9), s);  // + tile counters
    int hb = (n + 4 * kSortThreads - 1) / (4 * kSortThreads);
    if (hb > 2 * 152) hb = 2 * 152;
    k_sort_hist_all<<<hb > 0 ? hb : 1, kSortThreads, 0, s>>>(key[0], n, sc.ghist);
    k_sort_offsets<<<1, kRadix, 0, s>>>(sc.ghist, sc.goff, sc.epoch);
    int* tiles = reinterpret_cast<int*>(sc.ghist + 8 * kRadix);
    int cur = 0;
    for (int p = 0; p < 8; ++p) {
        k_onesweep<<<nb, kSortThreads, 0, s>>>(key[cur], val[cur], key[cur ^ 1], val[cur ^ 1], n,
                                               8 * p, sc.goff + p * kRadix,
                                               sc.status + (size_t)p * nb * kRadix, tiles + p,
                                               sc.epoch, (unsigned int)p, sc.err, kSortSpinLimit,
                                               nullptr);
        cur ^= 1;
    }
    if (n_clouds > 1) {
        // a ninth stable pass by cloud: (cloud, key) order, each cloud back in its
        // fixed segment; the offsets of a cloud are its segment start
        k_onesweep<<<nb, kSortThreads, 0, s>>>(key[cur], val[cur], key[cur ^ 1], val[cur ^ 1], n,
                                               0, reinterpret_cast<const unsigned int*>(cloud_start),
                                               sc.status + (size_t)8 * nb * kRadix, tiles + 8,
                                               sc.epoch, 8u, sc.err, kSortSpinLimit, cloud);
        cur ^= 1;
    }
    k_tiefix<<<(n + 255) / 256, 256, 0, s>>>(key[cur], val[cur], ids_in, n);
    return cur;
}

int sort_selftest_timeout(SortScratch sc, cudaStream_t s)
{
    // a lone block that takes tile 1 while tile 0 never publishes: its bounded
    // wait must run out, raise *err and leave the keys where they are
    count_launch(1);
    static const int one = 1;
    int* tiles = reinterpret_cast<int*>(sc.ghist + 8 * kRadix);
    if (cudaMemsetAsync(sc.status, 0, sizeof(unsigned long long) * 2 * kRadix, s) != cudaSuccess ||
        cudaMemcpyAsync(tiles, &one, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(sc.goff, 0, sizeof(unsigned int) * kRadix, s) != cudaSuccess ||
        cudaMemcpyAsync(sc.test_epoch, &one, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(sc.test_keys, 0, sizeof(unsigned long long) * 4 * kSortTile, s) != cudaSuccess ||
        cudaMemsetAsync(sc.test_vals, 0, sizeof(unsigned int) * 4 * kSortTile, s) != cudaSuccess)
        return -1;
    // input: tiles 0-1 of the test buffers; output: tiles 2-3
    k_onesweep<<<1, kSortThreads, 0, s>>>(sc.test_keys, sc.test_vals, sc.test_keys + 2 * kSortTile,
                                          sc.test_vals + 2 * kSortTile, 2 * kSortTile, 0, sc.goff,
                                          sc.status, tiles, sc.test_epoch, 0u, sc.err, 2000, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_tiefix(const unsigned long long* key, unsigned int* perm, const unsigned int* ids,
                   int n, cudaStream_t s)
{
    count_launch(1);
    k_tiefix<<<(n + 255) / 256, 256, 0, s>>>(key, perm, ids, n);
}

void launch_topology(const unsigned long long* key, int n, int leaf_cap, int* pos_cnt,
                     int* pos_off, int* scan_part, Tree t, cudaStream_t s)
{
    count_launch(3);
    cudaMemsetAsync(t.maxdepth, 0, sizeof(int), s);
    cudaMemsetAsync(t.count, 0, sizeof(int) * (kMaxDepth + 2), s);
    const int nb = (n + kTopoThreads - 1) / kTopoThreads;
    const bool win = leaf_cap <= kTopoWin;
    if (win) k_topo_count_win<<<nb, kTopoThreads, 0, s>>>(key, n, leaf_cap, pos_cnt, t);
    else k_topo_count<<<nb, kTopoThreads, 0, s>>>(key, n, leaf_cap, pos_cnt, t);
    launch_scan(pos_cnt, pos_off, n, scan_part, t.nnodes, s);
    k_clear_children<<<2 * 152, 256, 0, s>>>(t);
    if (win) k_topo_emit<true><<<nb, kTopoThreads, 0, s>>>(key, n, leaf_cap, pos_cnt, pos_off, t);
    else k_topo_emit<false><<<nb, kTopoThreads, 0, s>>>(key, n, leaf_cap, pos_cnt, pos_off, t);
}

void launch_moments(const double* x, const double* y, const double* z, const int8_t* sp,
                    const double* qsp, int n, const Cube* cube, Tree t, float4* src32,
                    int want_f32, cudaStream_t s)
{
    // leaves from their particles, then every twig as its last child finishes
    // (bottom-up sweep with arrival counters), in one launch
    count_launch(1);
    cudaMemsetAsync(t.arrive, 0, sizeof(int) * (size_t)t.cap, s);
    // small blocks spread the leaf threads (about one per eight particles) evenly
    // over the SMs
    int blocks = (n + kMomThreads - 1) / kMomThreads;
    if (blocks > 16 * 152) blocks = 16 * 152;
    if (blocks < 1) blocks = 1;
    if (want_f32)
        k_moments_leaves_f32<<<blocks, kMomThreads, 0, s>>>(x, y, z, sp, qsp, cube, t, src32);
    else
        k_moments_leaves<<<blocks, kMomThreads, 0, s>>>(x, y, z, sp, qsp, cube, t, src32, 0);
}

}  // namespace ucp
