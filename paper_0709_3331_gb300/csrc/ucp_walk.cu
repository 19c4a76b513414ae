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
// "next", no stack).  The walk writes (box, lane mask) entries into per-warp
// interaction lists in shared memory; full lists are evaluated in bulk, so the
// multipole and pair loops run without divergence.  Each lane sums its own
// target in a fixed order, so results do not depend on scheduling.
#include "ucp_internal.cuh"

#include <math.h>

namespace ucp {

namespace {

constexpr int kWalkThreads = 128;
constexpr int kWalkWarps = kWalkThreads / 32;
constexpr int kList = 64;

struct WarpLists {
    int m2p_node[kList];
    unsigned int m2p_mask[kList];
    int p2p_node[kList];
    unsigned int p2p_mask[kList];
};

__device__ __forceinline__ int next_chunk(int* work, int lane)
{
    int c = 0;
    if (lane == 0) c = atomicAdd(work, 1);
    return __shfl_sync(0xffffffffu, c, 0);
}

// ------------------------------------------------------------------ FP64
// Field of a box's expansion at R = x_t - c (softened kernel g = (R^2+eps^2)^-1/2):
//   E = M R g^3 - D g^3 + 3 (D.R) R g^5 - 3 (Q R) g^5 + 15/2 (R.Q.R) R g^7 - 3/2 tr(Q) R g^5
//   phi = M g + (D.R) g^3 + 1/2 (3 R.Q.R g^5 - tr(Q) g^3)
__device__ __forceinline__ void m2p_fp64(const double* __restrict__ m, double rx, double ry,
                                         double rz, double eps2, double& ex, double& ey,
                                         double& ez, double& ph)
{
    double M = m[MM];
    double Dx = m[MD], Dy = m[MD + 1], Dz = m[MD + 2];
    double Qxx = m[MQ], Qxy = m[MQ + 1], Qxz = m[MQ + 2], Qyy = m[MQ + 3], Qyz = m[MQ + 4],
           Qzz = m[MQ + 5];
    double r2 = rx * rx + ry * ry + rz * rz + eps2;
    double g = rsqrt(r2);
    double g2 = g * g;
    double g3 = g * g2, g5 = g3 * g2, g7 = g5 * g2;
    double DR = Dx * rx + Dy * ry + Dz * rz;
    double QRx = Qxx * rx + Qxy * ry + Qxz * rz;
    double QRy = Qxy * rx + Qyy * ry + Qyz * rz;
    double QRz = Qxz * rx + Qyz * ry + Qzz * rz;
    double RQR = rx * QRx + ry * QRy + rz * QRz;
    double trQ = Qxx + Qyy + Qzz;
    double a = M * g3 + 3.0 * DR * g5 + 7.5 * RQR * g7 - 1.5 * trQ * g5;
    double b = 3.0 * g5;
    ex += a * rx - Dx * g3 - b * QRx;
    ey += a * ry - Dy * g3 - b * QRy;
    ez += a * rz - Dz * g3 - b * QRz;
    ph += M * g + DR * g3 + 0.5 * (3.0 * RQR * g5 - trQ * g3);
}

__global__ void __launch_bounds__(kWalkThreads)
k_walk_fp64(WalkArgs a)
{
    __shared__ WarpLists L[kWalkWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpLists& lst = L[w];
    const int nn = *a.t.nnodes;
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const double* __restrict__ mom = a.t.mom;
    const int4* __restrict__ info = a.t.info;
    const int* __restrict__ dlf = a.t.depth_leaf;
    const double* __restrict__ X = a.x;
    const double* __restrict__ Y = a.y;
    const double* __restrict__ Z = a.z;
    const int8_t* __restrict__ SP = a.sp;

    for (int chunk = next_chunk(a.work, lane); chunk * 32 < a.ntargets;
         chunk = next_chunk(a.work, lane)) {
        const int ti = chunk * 32 + lane;
        const bool valid = ti < a.ntargets;
        const int t = valid ? (a.targets ? a.targets[ti] : ti) : -1;
        const double xt = valid ? X[t] : 0.0, yt = valid ? Y[t] : 0.0, zt = valid ? Z[t] : 0.0;
        double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
        int np = 0, nm = 0;
        int skip = valid ? 0 : 0x7fffffff;
        int nml = 0, npl = 0;

        auto flush = [&]() {
            __syncwarp();
            for (int e = 0; e < nml; ++e) {
                int nd = lst.m2p_node[e];
                if ((lst.m2p_mask[e] >> lane) & 1u) {
                    const double* m = mom + (size_t)nd * kMom;
                    m2p_fp64(m, xt - m[0], yt - m[1], zt - m[2], a.eps2, ex, ey, ez, ph);
                    ++nm;
                }
            }
            for (int e = 0; e < npl; ++e) {
                int nd = lst.p2p_node[e];
                if ((lst.p2p_mask[e] >> lane) & 1u) {
                    int4 inf = info[nd];
                    for (int j = inf.x; j < inf.y; ++j) {
                        if (j == t) continue;
                        double qj = SP[j] ? q1 : q0;
                        double dx = xt - X[j], dy = yt - Y[j], dz = zt - Z[j];
                        double r2 = dx * dx + dy * dy + dz * dz + a.eps2;
                        double ri = rsqrt(r2);
                        double qr3 = qj * ri * ri * ri;
                        ex += qr3 * dx;
                        ey += qr3 * dy;
                        ez += qr3 * dz;
                        ph += qj * ri;
                        ++np;
                    }
                }
            }
            nml = 0;
            npl = 0;
            __syncwarp();
        };

        int node = 0;
        while (node < nn) {
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
            const unsigned int am = __ballot_sync(0xffffffffu, acc);
            const unsigned int om = __ballot_sync(0xffffffffu, opn);
            if (am) {
                if (lane == 0) {
                    lst.m2p_node[nml] = node;
                    lst.m2p_mask[nml] = am;
                }
                ++nml;
            }
            if (om) {
                if (leaf) {
                    if (lane == 0) {
                        lst.p2p_node[npl] = node;
                        lst.p2p_mask[npl] = om;
                    }
                    ++npl;
                    node = inf.z;
                } else {
                    if (acc) skip = inf.z;
                    node = node + 1;
                }
            } else {
                node = inf.z;
            }
            if (nml == kList || npl == kList) flush();
        }
        flush();

        if (valid) {
            const int s = SP[t];
            const double qm = (s ? q1 : q0) / a.msp[s];
            a.ax[t] = qm * ex;
            a.ay[t] = qm * ey;
            a.az[t] = qm * ez;
            if (a.phi) a.phi[t] = ph;
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
// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v)
{
    float t = s + v;
    float bp = t - s;
    float ap = t - bp;
    c += (s - ap) + (v - bp);
    s = t;
}

__global__ void __launch_bounds__(kWalkThreads)
k_walk_fp32c(WalkArgs a)
{
    __shared__ WarpLists L[kWalkWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpLists& lst = L[w];
    const int nn = *a.t.nnodes;
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const float4* __restrict__ F = a.t.f32;
    const float4* __restrict__ S = a.src32;
    const float eps2 = (float)a.eps2;

    for (int chunk = next_chunk(a.work, lane); chunk * 32 < a.ntargets;
         chunk = next_chunk(a.work, lane)) {
        const int ti = chunk * 32 + lane;
        const bool valid = ti < a.ntargets;
        const int t = valid ? (a.targets ? a.targets[ti] : ti) : -1;
        // target as an unevaluated float pair: x = xh + xl
        float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f;
        if (valid) {
            double X = a.x[t], Y = a.y[t], Z = a.z[t];
            xh = (float)X; yh = (float)Y; zh = (float)Z;
            xl = (float)(X - (double)xh); yl = (float)(Y - (double)yh); zl = (float)(Z - (double)zh);
        }
        // compensated accumulators (sum, correction) for E and phi
        float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
        int np = 0, nm = 0;
        int skip = valid ? 0 : 0x7fffffff;
        int nml = 0, npl = 0;

        auto flush = [&]() {
            __syncwarp();
            float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
            for (int e = 0; e < nml; ++e) {
                int nd = lst.m2p_node[e];
                if ((lst.m2p_mask[e] >> lane) & 1u) {
                    const float4* r = F + (size_t)nd * kF32;
                    float4 A = r[0], B = r[1], C = r[2], D = r[3], E = r[4];
                    float rx = (xh - A.x) + (xl - B.x);
                    float ry = (yh - A.y) + (yl - B.y);
                    float rz = (zh - A.z) + (zl - B.z);
                    float M = C.z, Dx = C.w, Dy = D.x, Dz = D.y;
                    float Qxx = D.z, Qxy = D.w, Qxz = E.x, Qyy = E.y, Qyz = E.z, Qzz = E.w;
                    float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2)));
                    float g = rsqrtf(r2);
                    float g2 = g * g;
                    float g3 = g * g2, g5 = g3 * g2, g7 = g5 * g2;
                    float DR = fmaf(Dx, rx, fmaf(Dy, ry, Dz * rz));
                    float QRx = fmaf(Qxx, rx, fmaf(Qxy, ry, Qxz * rz));
                    float QRy = fmaf(Qxy, rx, fmaf(Qyy, ry, Qyz * rz));
                    float QRz = fmaf(Qxz, rx, fmaf(Qyz, ry, Qzz * rz));
                    float RQR = fmaf(rx, QRx, fmaf(ry, QRy, rz * QRz));
                    float trQ = Qxx + Qyy + Qzz;
                    float aa = fmaf(M, g3, fmaf(3.f * DR, g5, fmaf(7.5f * RQR, g7, -1.5f * trQ * g5)));
                    float b = 3.f * g5;
                    bx += fmaf(aa, rx, -fmaf(Dx, g3, b * QRx));
                    by += fmaf(aa, ry, -fmaf(Dy, g3, b * QRy));
                    bz += fmaf(aa, rz, -fmaf(Dz, g3, b * QRz));
                    bp += fmaf(M, g, fmaf(DR, g3, 0.5f * fmaf(3.f * RQR, g5, -trQ * g3)));
                    ++nm;
                }
            }
            two_sum_acc(sx, cx, bx);
            two_sum_acc(sy, cy, by);
            two_sum_acc(sz, cz, bz);
            two_sum_acc(sp, cp, bp);
            for (int e = 0; e < npl; ++e) {
                int nd = lst.p2p_node[e];
                if ((lst.p2p_mask[e] >> lane) & 1u) {
                    const float4* r = F + (size_t)nd * kF32;
                    float4 A = r[0], B = r[1], C = r[2];
                    float rx = (xh - A.x) + (xl - B.x);
                    float ry = (yh - A.y) + (yl - B.y);
                    float rz = (zh - A.z) + (zl - B.z);
                    int jb = __float_as_int(C.x), je = __float_as_int(C.y);
                    float px = 0.f, py = 0.f, pz = 0.f, pp = 0.f;
                    for (int j = jb; j < je; ++j) {
                        float4 s = __ldg(S + j);
                        float dx = rx - s.x, dy = ry - s.y, dz = rz - s.z;
                        float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                        float ri = (j == t) ? 0.f : rsqrtf(r2);
                        float qi = s.w * ri;
                        float qr3 = qi * ri * ri;
                        px = fmaf(qr3, dx, px);
                        py = fmaf(qr3, dy, py);
                        pz = fmaf(qr3, dz, pz);
                        pp += qi;
                    }
                    np += (je - jb) - ((t >= jb && t < je) ? 1 : 0);
                    two_sum_acc(sx, cx, px);
                    two_sum_acc(sy, cy, py);
                    two_sum_acc(sz, cz, pz);
                    two_sum_acc(sp, cp, pp);
                }
            }
            nml = 0;
            npl = 0;
            __syncwarp();
        };

        int node = 0;
        while (node < nn) {
            const float4* r = F + (size_t)node * kF32;
            const float4 A = r[0], B = r[1], C = r[2];
            const int nxt = __float_as_int(B.w);
            const bool leaf = __float_as_int(C.y) >= 0;
            const bool active = node >= skip;
            float rx = (xh - A.x) + (xl - B.x);
            float ry = (yh - A.y) + (yl - B.y);
            float rz = (zh - A.z) + (zl - B.z);
            float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            bool acc = active && (A.w < d2);
            // Within FP32 rounding of the threshold the decision is taken again in
            // FP64 exactly as the FP64 walk takes it, so both precisions open the
            // same boxes (rare: |d2 - rcrit2| <= 4e-6 d2).
            if (active && fabsf(d2 - A.w) <= 4e-6f * d2) {
                const double* m = a.t.mom + (size_t)node * kMom;
                double dx = __dsub_rn(a.x[t], m[0]);
                double dy = __dsub_rn(a.y[t], m[1]);
                double dz = __dsub_rn(a.z[t], m[2]);
                double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                      __dmul_rn(dz, dz));
                acc = m[MR2] < dd;
            }
            const bool opn = active && !acc;
            const unsigned int am = __ballot_sync(0xffffffffu, acc);
            const unsigned int om = __ballot_sync(0xffffffffu, opn);
            if (am) {
                if (lane == 0) {
                    lst.m2p_node[nml] = node;
                    lst.m2p_mask[nml] = am;
                }
                ++nml;
            }
            if (om) {
                if (leaf) {
                    if (lane == 0) {
                        lst.p2p_node[npl] = node;
                        lst.p2p_mask[npl] = om;
                    }
                    ++npl;
                    node = nxt;
                } else {
                    if (acc) skip = nxt;
                    node = node + 1;
                }
            } else {
                node = nxt;
            }
            if (nml == kList || npl == kList) flush();
        }
        flush();

        if (valid) {
            const int s = a.sp[t];
            const double qm = (s ? q1 : q0) / a.msp[s];
            a.ax[t] = qm * ((double)sx + (double)cx);
            a.ay[t] = qm * ((double)sy + (double)cy);
            a.az[t] = qm * ((double)sz + (double)cz);
            if (a.phi) a.phi[t] = (double)sp + (double)cp;
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
    const double L = cube->L;
    for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
        double* m = t.mom + (size_t)nd * kMom;
        int dl = t.depth_leaf[nd];
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
            float chx = (float)m[0], chy = (float)m[1], chz = (float)m[2];
            r[0] = make_float4(chx, chy, chz, (float)r2);
            r[1] = make_float4((float)(m[0] - (double)chx), (float)(m[1] - (double)chy),
                               (float)(m[2] - (double)chz), __int_as_float(inf.z));
            r[2] = make_float4(__int_as_float((dl & 256) ? inf.x : 0),
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

static int walk_blocks(int ntargets, int nsm, int per_sm)
{
    int chunks = (ntargets + 31) / 32;
    int blocks = nsm * per_sm;
    int need = (chunks + kWalkWarps - 1) / kWalkWarps;
    if (blocks > need) blocks = need;
    return blocks < 1 ? 1 : blocks;
}

void launch_walk_fp64(const WalkArgs& a, int nsm, cudaStream_t s)
{
    count_launch(1);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    k_walk_fp64<<<walk_blocks(a.ntargets, nsm, 8), kWalkThreads, 0, s>>>(a);
}

void launch_walk_fp32c(const WalkArgs& a, int nsm, cudaStream_t s)
{
    count_launch(1);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    k_walk_fp32c<<<walk_blocks(a.ntargets, nsm, 12), kWalkThreads, 0, s>>>(a);
}

}  // namespace ucp
