// ucp_walk.cu -- particle-TREE interaction of Sec. 3 (arXiv 0709.3331): for
// every target, boxes are visited from the root in pre-order; a box that
// satisfies the opening criterion of Eq. 5, s/theta + delta < d, acts through
// its expansion about its centroid (monopole, dipole, second moment of the
// softened kernel); an opened leaf is summed pair by pair.
//
// GPU form: one warp walks 32 key-consecutive targets (one per lane).  The
// per-target criterion is evaluated per lane; the warp descends into a box
// when any lane opens it, and a lane that accepted an ancestor sits out until
// the walk passes that ancestor's subtree (pre-order array with skip index
// "next", no stack).  Lanes that accept a box evaluate its expansion on the
// spot, reusing R = x_t - c and |R|^2 from the criterion; opened leaves go
// into a per-warp list in shared memory as (leaf, lane mask) and are summed in
// bulk, so the pair loop is warp-uniform.  Each lane sums its own target in a
// fixed order, so results do not depend on scheduling.
#include "ucp_internal.cuh"

#include <math.h>

namespace ucp {

namespace {

constexpr int kWalkThreads = 128;
constexpr int kList = 64;      // opened leaves buffered per warp
constexpr int kM2PBatch = 32;  // visits whose multipoles are summed in FP32 before a
                               // compensated add (a power of two)

struct WarpList {
    int leaf[kList];
    unsigned int mask[kList];
};

__device__ __forceinline__ int next_chunk(int* work, int lane)
{
    int c = 0;
    if (lane == 0) c = atomicAdd(work, 1);
    return __shfl_sync(0xffffffffu, c, 0);
}

// Error-free sum (Knuth's TwoSum) folded into a running correction.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v)
{
    float t = s + v;
    float bp = t - s;
    float ap = t - bp;
    c += (s - ap) + (v - bp);
    s = t;
}

// ---- bulk copies (TMA) of a leaf's sources into shared memory, completion
// tracked by an mbarrier (one arrival carrying the byte count)
__device__ __forceinline__ unsigned int smem_addr(const void* p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// generic-proxy reads of a buffer are ordered before the next bulk copy into it
__device__ __forceinline__ void async_proxy_fence()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned int bytes,
                                          unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned int parity)
{
    unsigned int ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
constexpr int kStagePairs = 16;          // sources staged per leaf: up to 32 (16 pairs)
constexpr int kStageSpin = 1 << 20;      // polls of a copy's barrier before giving up

// ------------------------------------------------------------------ FP64
// Expansion of a box at R = x_t - c, r2 = R.R + eps^2, g = r2^-1/2, u = g^2:
//   phi = g (M + u (D.R - tr(Q)/2 + (3/2) u R.Q.R))
//   E   = g^3 (M + 3u (D.R - tr(Q)/2 + (5/2) u R.Q.R)) R - g^3 (D + 3u Q R)
// (the Taylor expansion of the softened kernel through second order, with the
// terms of each power of u collected).
template <class T>
__device__ __forceinline__ void m2p(T rx, T ry, T rz, T r2, T M, T Dx, T Dy, T Dz, T Qxx, T Qxy,
                                    T Qxz, T Qyy, T Qyz, T Qzz, T& ex, T& ey, T& ez, T& ph);

template <>
__device__ __forceinline__ void m2p<double>(double rx, double ry, double rz, double r2, double M,
                                            double Dx, double Dy, double Dz, double Qxx,
                                            double Qxy, double Qxz, double Qyy, double Qyz,
                                            double Qzz, double& ex, double& ey, double& ez,
                                            double& ph)
{
    double g = rsqrt(r2);
    double u = g * g;
    double g3 = g * u;
    double QRx = Qxx * rx + Qxy * ry + Qxz * rz;
    double QRy = Qxy * rx + Qyy * ry + Qyz * rz;
    double QRz = Qxz * rx + Qyz * ry + Qzz * rz;
    double RQR = rx * QRx + ry * QRy + rz * QRz;
    double w = Dx * rx + Dy * ry + Dz * rz - 0.5 * (Qxx + Qyy + Qzz);
    double h = u * RQR;
    ph += g * (M + u * (w + 1.5 * h));
    double s3 = 3.0 * u;
    double aa = g3 * (M + s3 * (w + 2.5 * h));
    ex += aa * rx - g3 * (Dx + s3 * QRx);
    ey += aa * ry - g3 * (Dy + s3 * QRy);
    ez += aa * rz - g3 * (Dz + s3 * QRz);
}

// FP32 form; T = -tr(Q)/2 comes with the box record.  kPhi = false: field only.
template <bool kPhi>
__device__ __forceinline__ void m2p_f32(float rx, float ry, float rz, float r2, float T, float M,
                                        float Dx, float Dy, float Dz, float Qxx, float Qxy,
                                        float Qxz, float Qyy, float Qyz, float Qzz, float& ex,
                                        float& ey, float& ez, float& ph)
{
    float g = rsqrt_ftz(r2);
    float u = g * g;
    float g3 = g * u;
    float QRx = fmaf(Qxx, rx, fmaf(Qxy, ry, Qxz * rz));
    float QRy = fmaf(Qxy, rx, fmaf(Qyy, ry, Qyz * rz));
    float QRz = fmaf(Qxz, rx, fmaf(Qyz, ry, Qzz * rz));
    float RQR = fmaf(rx, QRx, fmaf(ry, QRy, rz * QRz));
    float w = fmaf(Dx, rx, fmaf(Dy, ry, fmaf(Dz, rz, T)));
    float h = u * RQR;
    if (kPhi) ph = fmaf(g, fmaf(u, fmaf(1.5f, h, w), M), ph);
    float s3 = 3.f * u;
    float aa = g3 * fmaf(s3, fmaf(2.5f, h, w), M);
    float mg3 = -g3;
    ex = fmaf(mg3, fmaf(s3, QRx, Dx), fmaf(aa, rx, ex));
    ey = fmaf(mg3, fmaf(s3, QRy, Dy), fmaf(aa, ry, ey));
    ez = fmaf(mg3, fmaf(s3, QRz, Dz), fmaf(aa, rz, ez));
}

template <bool kKelbg, int kThreads>
__global__ void __launch_bounds__(kThreads)
k_walk_fp64(WalkArgs a)
{
    __shared__ WarpList L[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpList& lst = L[w];
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const double* __restrict__ mom = a.t.mom;
    const int4* __restrict__ info = a.t.info;
    const int* __restrict__ dlf = a.t.depth_leaf;
    const double* __restrict__ X = a.x;
    const double* __restrict__ Y = a.y;
    const double* __restrict__ Z = a.z;
    const int8_t* __restrict__ SP = a.sp;

    for (int chunk = next_chunk(a.work, lane); chunk < a.nchunks;
         chunk = next_chunk(a.work, lane)) {
        // up to 32 key-consecutive targets of one cloud, walked through that cloud's tree
        const int4 ck = a.chunks[chunk];
        const int ti = ck.x + lane;
        const bool valid = lane < ck.y;
        const int t = valid ? (a.targets ? a.targets[ti] : ti) : -1;
        const int root = a.pos_off[a.t.cloud_start ? a.t.cloud_start[ck.z] : 0];
        const int end = info[root].z;
        const double xt = valid ? X[t] : 0.0, yt = valid ? Y[t] : 0.0, zt = valid ? Z[t] : 0.0;
        const int8_t st = valid ? SP[t] : 0;
        // multipole and direct-pair sums kept apart: each is then a sum over this
        // target's own boxes in pre-order, whichever targets share the warp
        double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
        double pex = 0.0, pey = 0.0, pez = 0.0, pph = 0.0;
        int np = 0, nm = 0;
        int skip = valid ? 0 : 0x7fffffff;
        int npl = 0;

        auto flush = [&]() {
            __syncwarp();
            for (int e = 0; e < npl; ++e) {
                int nd = lst.leaf[e];
                if ((lst.mask[e] >> lane) & 1u) {
                    int4 inf = info[nd];
                    for (int j = inf.x; j < inf.y; ++j) {
                        if (j == t) continue;
                        double qj = SP[j] ? q1 : q0;
                        double dx = xt - X[j], dy = yt - Y[j], dz = zt - Z[j];
                        if (kKelbg && SP[j] != st) {
                            // Sec. 2.1 Eq. 3: qj (1 - e)/r, e = exp(-r/lambda);
                            // E = qj r_vec [(1 - e)/r^3 - e/(lambda r^2)]
                            double r = sqrt(dx * dx + dy * dy + dz * dz);
                            ++np;
                            if (r == 0.0) {
                                pph += qj / a.lambda;
                                continue;
                            }
                            double u = r / a.lambda;
                            double e = exp(-u), ome = -expm1(-u);
                            double f = ome / (r * r * r) - e / (a.lambda * r * r);
                            pex += qj * dx * f;
                            pey += qj * dy * f;
                            pez += qj * dz * f;
                            pph += qj * ome / r;
                            continue;
                        }
                        double r2 = dx * dx + dy * dy + dz * dz + a.eps2;
                        double ri = rsqrt(r2);
                        double qr3 = qj * ri * ri * ri;
                        pex += qr3 * dx;
                        pey += qr3 * dy;
                        pez += qr3 * dz;
                        pph += qj * ri;
                        ++np;
                    }
                }
            }
            npl = 0;
            __syncwarp();
        };

        int node = root;
        while (node < end) {
            const double* m = mom + (size_t)node * kMom;
            const int4 inf = info[node];
            const bool leaf = (dlf[node] & 256) != 0;
            const bool active = node >= skip;
            // Eq. 5 as (s/theta + delta)^2 < |x_t - c|^2, rounded like the definition
            double dx = __dsub_rn(xt, m[0]);
            double dy = __dsub_rn(yt, m[1]);
            double dz = __dsub_rn(zt, m[2]);
            double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                  __dmul_rn(dz, dz));
            const bool acc = active && (m[MR2] < d2);
            const bool opn = active && !acc;
            const unsigned int om = __ballot_sync(0xffffffffu, opn);
            int next = inf.z;
            if (om) {
                if (leaf) {
                    if (lane == 0) {
                        lst.leaf[npl] = node;
                        lst.mask[npl] = om;
                    }
                    ++npl;
                } else {
                    if (acc) skip = inf.z;
                    next = node + 1;
                }
            }
            if (acc) {
                m2p<double>(dx, dy, dz, d2 + a.eps2, m[MM], m[MD], m[MD + 1], m[MD + 2], m[MQ],
                            m[MQ + 1], m[MQ + 2], m[MQ + 3], m[MQ + 4], m[MQ + 5], ex, ey, ez, ph);
                ++nm;
            }
            node = next;
            if (npl == kList) flush();
        }
        flush();

        if (valid) {
            const int s = SP[t];
            const double qm = (s ? q1 : q0) / a.msp[s];
            a.ax[t] = qm * (ex + pex);
            a.ay[t] = qm * (ey + pey);
            a.az[t] = qm * (ez + pez);
            if (a.phi) a.phi[t] = ph + pph;
            a.cnt_p2p[t] = np;
            a.cnt_m2p[t] = nm;
        }
        unsigned long long sp2 = (unsigned long long)np, sm2 = (unsigned long long)nm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp2 += __shfl_xor_sync(0xffffffffu, sp2, o);
            sm2 += __shfl_xor_sync(0xffffffffu, sm2, o);
        }
        if (lane == 0) {
            atomicAdd(&a.stats[0], sp2);
            atomicAdd(&a.stats[1], sm2);
        }
    }
}

// ------------------------------------------------------------------ FP32C
// Kelbg pair factors in FP32 for u = r/lambda: p = (1 - e^-u)/u and
// g = (1 - (1 + u) e^-u)/u^3, by their Taylor series below u = 1/2 (no
// cancellation) and directly above.
__device__ __forceinline__ void kelbg_pg(float u, float& p, float& g)
{
    if (u < 0.5f) {
        p = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, 1.f / 5040.f, -1.f / 720.f),
                                                    1.f / 120.f), -1.f / 24.f), 1.f / 6.f),
                          -0.5f), 1.f);
        float poly = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, 1.f / 5760.f, -1.f / 840.f),
                                                  1.f / 144.f), -1.f / 30.f), 0.125f),
                          -1.f / 3.f);
        g = 0.5f / u + poly;
    } else {
        float e = __expf(-u);
        float iu = 1.f / u;
        p = (1.f - e) * iu;
        g = (1.f - (1.f + u) * e) * iu * iu * iu;
    }
}

// kThreads threads per block, register budget for kBlocks resident blocks per SM.
// kStage: a leaf's sources (up to 32) are brought into shared memory by a bulk
// copy issued one list entry ahead (double buffer per warp) instead of being read
// through L1 by every lane; the arithmetic and its order are the same.
// kPhi = false (walks whose potential nobody reads, e.g. the electron substeps):
// the potential terms and their sums are left out; the field is computed by the
// same operations in the same order, so accelerations are bit-identical.
template <bool kKelbg, int kThreads, int kBlocks, bool kStage, bool kPhi>
__global__ void __launch_bounds__(kThreads, kBlocks)
k_walk_fp32c(WalkArgs a)
{
    __shared__ WarpList L[kThreads / 32];
    __shared__ __align__(16) float4 stage[kStage ? kThreads / 32 : 1][2][2 * kStagePairs];
    __shared__ __align__(8) unsigned long long stage_bar[kStage ? kThreads / 32 : 1][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpList& lst = L[w];
    unsigned int stage_phase = 0;  // parity to wait for, per buffer (bits 0, 1)
    bool stage_ok = kStage;        // cleared for good if a copy is not seen to complete
    if (kStage) {
        if (lane == 0) {
            mbar_init(&stage_bar[w][0]);
            mbar_init(&stage_bar[w][1]);
            mbar_init_fence();
        }
        __syncwarp();
    }
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const float4* __restrict__ F = a.t.f32;
    const float4* __restrict__ S = a.src32;
    const float eps2 = (float)a.eps2;

    for (int chunk = next_chunk(a.work, lane); chunk < a.nchunks;
         chunk = next_chunk(a.work, lane)) {
        // up to 32 key-consecutive targets of one cloud, walked through that cloud's tree
        const int4 ck = a.chunks[chunk];
        const int ti = ck.x + lane;
        const bool valid = lane < ck.y;
        const int t = valid ? (a.targets ? a.targets[ti] : ti) : -1;
        const int root = a.pos_off[a.t.cloud_start ? a.t.cloud_start[ck.z] : 0];
        const int end = __float_as_int(F[(size_t)root * kF32 + 1].w);
        // target as an unevaluated float pair: x = xh + xl ({x, y} packed for the
        // FP32x2 adds), relative to the centre of the cloud's cube like the box
        // centroids, so that the FP32 errors scale with the cloud's size and not
        // with its distance from the origin
        float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f;
        if (valid) {
            const double* cc = a.cubes[ck.z].c;
            double X = a.x[t] - cc[0], Y = a.y[t] - cc[1], Z = a.z[t] - cc[2];
            xh = (float)X; yh = (float)Y; zh = (float)Z;
            xl = (float)(X - (double)xh); yl = (float)(Y - (double)yh); zl = (float)(Z - (double)zh);
        }
        const float2 xyh = make_float2(xh, yh);
        // Window of the FP32 criterion (see the traversal): |dm| <= wa d2 + wb
        // bounds the FP32 error of d2 - rcrit2 for this target, given
        // |x_t - xh| <= 2^-24 |x_t| and the same for the centroid
        const float bt = 5e-7f * fmaxf(fabsf(xh), fmaxf(fabsf(yh), fabsf(zh)));
        const float wa = fmaf(0.5f, bt, 4e-6f), wb = 0.5f * bt;
        const float qt = valid ? (a.sp[t] ? (float)q1 : (float)q0) : 0.f;
        const float inv_lambda = (float)(1.0 / a.lambda);
        const float inv_lambda3 = inv_lambda * inv_lambda * inv_lambda;
        // compensated totals (sum, correction) and the current multipole batch
        float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
        float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
        int np = 0, nm = 0, vis = 0;
        int skip = valid ? 0 : 0x7fffffff;
        int npl = 0;

        auto fold_batch = [&]() {
            two_sum_acc(sx, cx, bx);
            two_sum_acc(sy, cy, by);
            two_sum_acc(sz, cz, bz);
            if (kPhi) two_sum_acc(sp, cp, bp);
            bx = by = bz = bp = 0.f;
        };

        // one list entry's pair sum from sources at P0 (paired float4, P0[0] = the
        // pair that holds source jb)
        auto leaf_pairs = [&](int nd, const float4* __restrict__ P0) {
            const float4* r = F + (size_t)nd * kF32;
            float4 A = r[0], B = r[1], C = r[2];
            float rx = (xh + A.x) + (xl + B.x);
            float ry = (yh + A.y) + (yl + B.y);
            float rz = (zh + A.z) + (zl + B.z);
            int jb = __ldg(&a.t.info[nd].x), je = __float_as_int(C.y);
            const float2 rx2 = make_float2(rx, rx), ry2 = make_float2(ry, ry),
                         rz2 = make_float2(rz, rz), e2 = make_float2(eps2, eps2);
            float2 px = make_float2(0.f, 0.f), py = px, pz = px, pp = px;
#pragma unroll 2
            for (int j = jb & ~1; j < je; j += 2) {
                const float4 P = P0[j - (jb & ~1)], Q = P0[j - (jb & ~1) + 1];
                float2 dx = __fadd2_rn(rx2, make_float2(P.x, P.y));
                float2 dy = __fadd2_rn(ry2, make_float2(P.z, P.w));
                float2 dz = __fadd2_rn(rz2, make_float2(Q.x, Q.y));
                float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                const bool ok0 = j >= jb && j != t;
                const bool ok1 = j + 1 < je && j + 1 != t;
                float2 ri = make_float2(ok0 ? rsqrt_ftz(r2.x) : 0.f, ok1 ? rsqrt_ftz(r2.y) : 0.f);
                float2 qi = __fmul2_rn(make_float2(Q.z, Q.w), ri);
                float2 qr3 = __fmul2_rn(__fmul2_rn(qi, ri), ri);
                px = __ffma2_rn(qr3, dx, px);
                py = __ffma2_rn(qr3, dy, py);
                pz = __ffma2_rn(qr3, dz, pz);
                if (kPhi) pp = __fadd2_rn(pp, qi);
            }
            np += (je - jb) - ((t >= jb && t < je) ? 1 : 0);
            two_sum_acc(sx, cx, px.x + px.y);
            two_sum_acc(sy, cy, py.x + py.y);
            two_sum_acc(sz, cz, pz.x + pz.y);
            if (kPhi) two_sum_acc(sp, cp, pp.x + pp.y);
        };

        // Staged form: entry e's sources go to buffer e & 1 while entry e - 1 is
        // summed; entries with more than 32 sources read them from global memory.
        auto stage_entry = [&](int e) -> bool {
            const int nd = lst.leaf[e];
            const int jb = __ldg(&a.t.info[nd].x);
            const int je = __float_as_int(__ldg(&F[(size_t)nd * kF32 + 2]).y);
            const int pb = jb >> 1, pe = (je + 1) >> 1;
            if (!stage_ok || pe - pb > kStagePairs) return false;
            if (lane == 0) {
                async_proxy_fence();
                bulk_load(&stage[w][e & 1][0], S + 2 * (size_t)pb,
                          (unsigned int)(pe - pb) * 32u, &stage_bar[w][e & 1]);
            }
            return true;
        };
        auto flush_staged = [&]() {
            __syncwarp();
            bool st_cur = npl > 0 ? stage_entry(0) : false;
            for (int e = 0; e < npl; ++e) {
                bool st_next = e + 1 < npl ? stage_entry(e + 1) : false;
                const int nd = lst.leaf[e];
                const float4* P0;
                if (st_cur) {
                    const int b = e & 1;
                    const unsigned int par = (stage_phase >> b) & 1u;
                    bool done = false;
                    for (int it = 0; it < kStageSpin && !done; ++it)
                        done = mbar_test(&stage_bar[w][b], par);
                    stage_phase ^= 1u << b;
                    P0 = &stage[w][b][0];
                    if (!done) {
                        // raise the flag, stop staging in this warp and read this
                        // entry from global memory; the copies still in flight into
                        // this warp's buffers (this entry's, and the next entry's if
                        // it was issued) get one more bounded wait each, so that none
                        // lands after the warp has moved on
                        if (lane == 0) atomicExch(a.err, 1);
                        bool late = false;
                        for (int it = 0; it < kStageSpin && !late; ++it)
                            late = mbar_test(&stage_bar[w][b], par);
                        if (st_next) {
                            const int b1 = b ^ 1;
                            const unsigned int par1 = (stage_phase >> b1) & 1u;
                            late = false;
                            for (int it = 0; it < kStageSpin && !late; ++it)
                                late = mbar_test(&stage_bar[w][b1], par1);
                        }
                        stage_ok = false;
                        st_next = false;
                        P0 = S + ((size_t)__ldg(&a.t.info[nd].x) & ~(size_t)1);
                    }
                } else {
                    P0 = S + ((size_t)__ldg(&a.t.info[nd].x) & ~(size_t)1);
                }
                if ((lst.mask[e] >> lane) & 1u) leaf_pairs(nd, P0);
                __syncwarp();
                st_cur = st_next;
            }
            npl = 0;
            __syncwarp();
        };

        auto flush = [&]() {
            if (kStage && !kKelbg) {
                flush_staged();
                return;
            }
            __syncwarp();
            for (int e = 0; e < npl; ++e) {
                int nd = lst.leaf[e];
                if ((lst.mask[e] >> lane) & 1u) {
                    const float4* r = F + (size_t)nd * kF32;
                    float4 A = r[0], B = r[1], C = r[2];
                    float rx = (xh + A.x) + (xl + B.x);
                    float ry = (yh + A.y) + (yl + B.y);
                    float rz = (zh + A.z) + (zl + B.z);
                    int jb = __ldg(&a.t.info[nd].x), je = __float_as_int(C.y);
                    if (kKelbg) {
                        // one source at a time: unlike charges (electron-ion) take the
                        // Kelbg form, like charges the softened Coulomb law
                        float px = 0.f, py = 0.f, pz = 0.f, pp = 0.f;
                        for (int j = jb; j < je; ++j) {
                            if (j == t) continue;
                            const float4 P = __ldg(S + (j & ~1)), Q = __ldg(S + (j & ~1) + 1);
                            const bool odd = j & 1;
                            float dx = rx + (odd ? P.y : P.x);
                            float dy = ry + (odd ? P.w : P.z);
                            float dz = rz + (odd ? Q.y : Q.x);
                            float qj = odd ? Q.w : Q.z;
                            if (qj != qt) {
                                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                if (r2 == 0.f) {
                                    pp = fmaf(qj, inv_lambda, pp);
                                    continue;
                                }
                                float r = sqrtf(r2);
                                float pf, gf;
                                kelbg_pg(r * inv_lambda, pf, gf);
                                float fq = qj * gf * inv_lambda3;
                                px = fmaf(fq, dx, px);
                                py = fmaf(fq, dy, py);
                                pz = fmaf(fq, dz, pz);
                                pp = fmaf(qj * inv_lambda, pf, pp);
                            } else {
                                float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                                float ri = rsqrt_ftz(r2);
                                float qi = qj * ri;
                                float qr3 = qi * ri * ri;
                                px = fmaf(qr3, dx, px);
                                py = fmaf(qr3, dy, py);
                                pz = fmaf(qr3, dz, pz);
                                pp += qi;
                            }
                        }
                        np += (je - jb) - ((t >= jb && t < je) ? 1 : 0);
                        two_sum_acc(sx, cx, px);
                        two_sum_acc(sy, cy, py);
                        two_sum_acc(sz, cz, pz);
                        two_sum_acc(sp, cp, pp);
                        continue;
                    }
                    // sources in pairs {x_2p, x_2p+1, y.., y..}, {z.., z.., q.., q..} as
                    // offsets c_leaf - x_j; a pair member outside [jb, je) or equal to
                    // the target gets a zero inverse distance
                    const float2 rx2 = make_float2(rx, rx), ry2 = make_float2(ry, ry),
                                 rz2 = make_float2(rz, rz), e2 = make_float2(eps2, eps2);
                    float2 px = make_float2(0.f, 0.f), py = px, pz = px, pp = px;
#pragma unroll 2
                    for (int j = jb & ~1; j < je; j += 2) {
                        const float4 P = __ldg(S + j), Q = __ldg(S + j + 1);
                        float2 dx = __fadd2_rn(rx2, make_float2(P.x, P.y));
                        float2 dy = __fadd2_rn(ry2, make_float2(P.z, P.w));
                        float2 dz = __fadd2_rn(rz2, make_float2(Q.x, Q.y));
                        float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                        const bool ok0 = j >= jb && j != t;
                        const bool ok1 = j + 1 < je && j + 1 != t;
                        float2 ri = make_float2(ok0 ? rsqrt_ftz(r2.x) : 0.f, ok1 ? rsqrt_ftz(r2.y) : 0.f);
                        float2 qi = __fmul2_rn(make_float2(Q.z, Q.w), ri);
                        float2 qr3 = __fmul2_rn(__fmul2_rn(qi, ri), ri);
                        px = __ffma2_rn(qr3, dx, px);
                        py = __ffma2_rn(qr3, dy, py);
                        pz = __ffma2_rn(qr3, dz, pz);
                        if (kPhi) pp = __fadd2_rn(pp, qi);
                    }
                    np += (je - jb) - ((t >= jb && t < je) ? 1 : 0);
                    two_sum_acc(sx, cx, px.x + px.y);
                    two_sum_acc(sy, cy, py.x + py.y);
                    two_sum_acc(sz, cz, pz.x + pz.y);
                    if (kPhi) two_sum_acc(sp, cp, pp.x + pp.y);
                }
            }
            npl = 0;
            __syncwarp();
        };

        int node = root;
        while (node < end) {
            const float4* r = F + (size_t)node * kF32;
            const float4 A = r[0], B = r[1], C = r[2], D = r[3], E = r[4];
            const int nxt = __float_as_int(B.w);
            const bool leaf = __float_as_int(C.y) >= 0;
            const bool active = node >= skip;
            // R = x_t - c from the rounded target and centroid (their low parts
            // enter only the direct pairs): one add per axis on the chain
            // record -> criterion -> vote -> next box that sets the walk's pace
            const float2 rxy = __fadd2_rn(xyh, make_float2(A.x, A.y));
            const float rx = rxy.x, ry = rxy.y;
            const float rz = zh + A.z;
            float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            const float dm = d2 - A.w;
            bool acc = active && dm > 0.f;
            // Within the FP32 error of d2 - rcrit2 the decision is taken again in
            // FP64 exactly as the FP64 walk takes it, so both precisions open the
            // same boxes.  Per axis R is off by at most 2^-23 (|x_t| + |R|), so
            // |error| <= 2^-22 sqrt(3) X_t d + 2^-21 d2 (rcrit2's rounding
            // included) with X_t the target's largest coordinate; with
            // d <= (d2 + 1) / 2 that lies inside wa d2 + wb (rare: a few tests in
            // a million at the bench size).
            if (active && fabsf(dm) <= fmaf(wa, d2, wb)) {
                const double* m = a.t.mom + (size_t)node * kMom;
                double dx = __dsub_rn(a.x[t], m[0]);
                double dy = __dsub_rn(a.y[t], m[1]);
                double dz = __dsub_rn(a.z[t], m[2]);
                double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                      __dmul_rn(dz, dz));
                acc = m[MR2] < dd;
            }
            const bool opn = active && !acc;
            const unsigned int om = __ballot_sync(0xffffffffu, opn);
            int next = nxt;
            if (om) {
                if (leaf) {
                    if (lane == 0) {
                        lst.leaf[npl] = node;
                        lst.mask[npl] = om;
                    }
                    ++npl;
                } else {
                    if (acc) skip = nxt;
                    next = node + 1;
                }
            }
            if (acc) {
                m2p_f32<kPhi>(rx, ry, rz, d2 + eps2, C.x, C.z, C.w, D.x, D.y, D.z, D.w, E.x, E.y, E.z,
                        E.w, bx, by, bz, bp);
                ++nm;
            }
            if ((++vis & (kM2PBatch - 1)) == 0) fold_batch();
            node = next;
            if (npl == kList) flush();
        }
        flush();
        fold_batch();

        if (valid) {
            const int s = a.sp[t];
            const double qm = (s ? q1 : q0) / a.msp[s];
            a.ax[t] = qm * ((double)sx + (double)cx);
            a.ay[t] = qm * ((double)sy + (double)cy);
            a.az[t] = qm * ((double)sz + (double)cz);
            if (kPhi && a.phi) a.phi[t] = (double)sp + (double)cp;
            a.cnt_p2p[t] = np;
            a.cnt_m2p[t] = nm;
        }
        unsigned long long sp2 = (unsigned long long)np, sm2 = (unsigned long long)nm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp2 += __shfl_xor_sync(0xffffffffu, sp2, o);
            sm2 += __shfl_xor_sync(0xffffffffu, sm2, o);
        }
        if (lane == 0) {
            atomicAdd(&a.stats[0], sp2);
            atomicAdd(&a.stats[1], sm2);
        }
    }
}

// Per walk: rcrit2 = (s/theta + delta)^2 of every box in FP64 (theta = 0:
// +inf, nothing accepted), and the FP32C box records.
__global__ void k_mac_prepare(Tree t, const Cube* __restrict__ cube, double theta, int want_f32)
{
    const int nn = *t.nnodes;
    for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
        double* m = t.mom + (size_t)nd * kMom;
        int dl = t.depth_leaf[nd];
        const Cube& cb = cube[t.cloud ? t.cloud[t.info[nd].x] : 0];
        const double L = cb.L;
        double s = ldexp(L, -(dl & 255));
        double r2;
        if (theta > 0.0) {
            double rc = __dadd_rn(__ddiv_rn(s, theta), m[MDELTA]);
            r2 = __dmul_rn(rc, rc);
        } else {
            r2 = INFINITY;
        }
        m[MR2] = r2;
        if (want_f32) {
            int4 inf = t.info[nd];
            float4* r = t.f32 + (size_t)nd * kF32;
            // the centroid, relative to the cube's centre as the walk's targets are,
            // enters negated (x_t - c as a sum); the trace term of the expansion as
            // one value
            const double ux = m[0] - cb.c[0], uy = m[1] - cb.c[1], uz = m[2] - cb.c[2];
            float chx = (float)ux, chy = (float)uy, chz = (float)uz;
            r[0] = make_float4(-chx, -chy, -chz, (float)r2);
            r[1] = make_float4((float)((double)chx - ux), (float)((double)chy - uy),
                               (float)((double)chz - uz), __int_as_float(inf.z));
            const float qxx = (float)m[MQ], qyy = (float)m[MQ + 3], qzz = (float)m[MQ + 5];
            r[2] = make_float4(-0.5f * ((qxx + qyy) + qzz),
                               __int_as_float((dl & 256) ? inf.y : -1), (float)m[MM],
                               (float)m[MD]);
            r[3] = make_float4((float)m[MD + 1], (float)m[MD + 2], (float)m[MQ], (float)m[MQ + 1]);
            r[4] = make_float4((float)m[MQ + 2], (float)m[MQ + 3], (float)m[MQ + 4],
                               (float)m[MQ + 5]);
        }
    }
}

}  // namespace

void launch_mac_prepare(Tree t, const Cube* cube, double theta, int want_f32, cudaStream_t s)
{
    count_launch(1);
    int blocks = 4 * 152;
    k_mac_prepare<<<blocks, 256, 0, s>>>(t, cube, theta, want_f32);
}

static int walk_blocks(int nchunks, int nsm, int per_sm, int warps_per_block)
{
    int blocks = nsm * per_sm;
    int need = (nchunks + warps_per_block - 1) / warps_per_block;
    if (blocks > need) blocks = need;
    return blocks < 1 ? 1 : blocks;
}

// Grid of th-thread blocks, per_sm resident per SM.  When the chunks cannot give
// every SM a block (small clouds), blocks narrow to one warp so the same warps
// spread over more SMs.  Each warp walks whole chunks, so no shape changes a result.
static void walk_grid(int nchunks, int nsm, int* th, int per_sm, int* blocks)
{
    const int wpb = *th / 32;
    *blocks = walk_blocks(nchunks, nsm, per_sm, wpb);
    if (*blocks < nsm && wpb > 1) {
        *th = 32;
        *blocks = walk_blocks(nchunks, nsm, per_sm * wpb, 1);
    }
}

void launch_walk_fp64(const WalkArgs& a, int nsm, cudaStream_t s)
{
    count_launch(1);
    int th = kWalkThreads, b;
    walk_grid(a.nchunks, nsm, &th, 8, &b);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    if (a.kelbg) {
        if (th == 32) k_walk_fp64<true, 32><<<b, 32, 0, s>>>(a);
        else k_walk_fp64<true, kWalkThreads><<<b, kWalkThreads, 0, s>>>(a);
    } else {
        if (th == 32) k_walk_fp64<false, 32><<<b, 32, 0, s>>>(a);
        else k_walk_fp64<false, kWalkThreads><<<b, kWalkThreads, 0, s>>>(a);
    }
}

// Launch shapes of the FP32C walk that the autotuner chooses from: threads per
// block, resident blocks per SM, which also sets the register budget (28 warps
// per SM at 72 registers, 32 at 64), and whether leaf sources are staged in
// shared memory by bulk copies.  The persistent grid takes 32-target
// chunks from a counter, so the shape changes the schedule, never a result.
static const int kShapes[][3] = {{128, 7, 0}, {896, 1, 0}, {128, 8, 0}, {1024, 1, 0},
                                 {256, 4, 0}, {512, 2, 0}, {128, 7, 1}, {896, 1, 1},
                                 {128, 8, 1}, {256, 4, 1}};
int walk_shape_count() { return (int)(sizeof(kShapes) / sizeof(kShapes[0])); }

template <bool kKelbg, bool kStage, bool kPhi>
static void walk_fp32c_shape(const WalkArgs& a, int th, int per_sm, int b, cudaStream_t s)
{
    if (th == 32) k_walk_fp32c<kKelbg, 32, 24, false, kPhi><<<b, 32, 0, s>>>(a);
    else if (th == 896) k_walk_fp32c<kKelbg, 896, 1, kStage, kPhi><<<b, 896, 0, s>>>(a);
    else if (th == 1024) k_walk_fp32c<kKelbg, 1024, 1, false, kPhi><<<b, 1024, 0, s>>>(a);
    else if (th == 256) k_walk_fp32c<kKelbg, 256, 4, kStage, kPhi><<<b, 256, 0, s>>>(a);
    else if (th == 512) k_walk_fp32c<kKelbg, 512, 2, false, kPhi><<<b, 512, 0, s>>>(a);
    else if (per_sm >= 8) k_walk_fp32c<kKelbg, 128, 8, kStage, kPhi><<<b, 128, 0, s>>>(a);
    else k_walk_fp32c<kKelbg, 128, 7, kStage, kPhi><<<b, 128, 0, s>>>(a);
}

void launch_walk_fp32c(const WalkArgs& a, int nsm, cudaStream_t s, int shape)
{
    count_launch(1);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    if (shape < 0 || shape >= walk_shape_count()) shape = 0;
    int th = kShapes[shape][0], b;
    const int per_sm = kShapes[shape][1];
    // the Kelbg pair law reads its sources directly
    const bool stage = kShapes[shape][2] != 0 && !a.kelbg;
    walk_grid(a.nchunks, nsm, &th, per_sm, &b);
    // the potential is computed only when the caller reads it (the Kelbg form
    // always computes it)
    const bool phi = a.phi != nullptr;
    if (a.kelbg) walk_fp32c_shape<true, false, true>(a, th, per_sm, b, s);
    else if (stage && phi) walk_fp32c_shape<false, true, true>(a, th, per_sm, b, s);
    else if (stage) walk_fp32c_shape<false, true, false>(a, th, per_sm, b, s);
    else if (phi) walk_fp32c_shape<false, false, true>(a, th, per_sm, b, s);
    else walk_fp32c_shape<false, false, false>(a, th, per_sm, b, s);
}

}  // namespace ucp
