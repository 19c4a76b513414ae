// ucp_adjoint.cu -- reverse-mode derivative of the TREE force of Sec. 3
// (arXiv 0709.3331): mu = (da/dx)^T lambda for a = q E / m with the tree held
// fixed (the boxes every target opens or accepts do not move under an
// infinitesimal displacement).  FP64.
//
// The walk visits exactly the boxes of the forward walk (same criterion, same
// rounding).  Per target (lane):
//   direct pair j:    mu_t += (q_t q_j / m_t) J(r) lambda_t,  J = g^3 I - 3 g^5 r r^T
//                     mu_j -= q_j J(r) w_t,  w_t = q_t lambda_t / m_t
//   accepted box n:   mu_t -= (q_t/m_t) (M d2g lambda - sum_bc lambda_b D_c d3g_abc
//                                        + 1/2 sum_bcd lambda_b Q_cd d4g_abcd)
//                     alpha_n += d2g w, Gamma_n += w_a d3g_a.., kappa_n += 1/2 d4g[w,.,Q]
// and afterwards every particle s of box n receives
//   q_s (alpha_n - Gamma_n (x_s - c_n)) + (|q_s| / S0_n) kappa_n
// (the source side through the dipole and second moment at fixed centre, and
// through the |q|-weighted centre the expansion is taken about).
// Source-side sums over targets are warp reductions followed by FP64 atomic
// adds, so their order (and last bits) may vary from run to run.
#include "ucp_internal.cuh"

#include <math.h>

namespace ucp {

namespace {

constexpr int kAdjThreads = 128;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjList = 64;

struct AdjList {
    int leaf[kAdjList];
    unsigned int mask[kAdjList];
};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double dot3(const double* a, const double* b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void qmul(const double* Q, const double* v, double* o)
{
    o[0] = Q[0] * v[0] + Q[1] * v[1] + Q[2] * v[2];
    o[1] = Q[1] * v[0] + Q[3] * v[1] + Q[4] * v[2];
    o[2] = Q[2] * v[0] + Q[4] * v[1] + Q[5] * v[2];
}

// sum_bcd v_b Q_cd d4g_abcd
__device__ __forceinline__ void t4(const double* R, const double* v, const double* Q, double g,
                                   double* o)
{
    double g2 = g * g, g5 = g2 * g2 * g, g7 = g5 * g2, g9 = g7 * g2;
    double QR[3], Qv[3];
    qmul(Q, R, QR);
    qmul(Q, v, Qv);
    double RQR = dot3(R, QR), Rv = dot3(R, v), vQR = dot3(v, QR), trQ = Q[0] + Q[3] + Q[5];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        o[a] = 105.0 * R[a] * Rv * RQR * g9 -
               15.0 * g7 * (v[a] * RQR + 2.0 * Rv * QR[a] + 2.0 * R[a] * vQR + R[a] * Rv * trQ) +
               3.0 * g5 * (v[a] * trQ + 2.0 * Qv[a]);
}

__global__ void __launch_bounds__(kAdjThreads)
k_walk_adjoint(WalkArgs a, const double* __restrict__ lam, double* __restrict__ mu,
               double* __restrict__ adj)
{
    __shared__ AdjList Ls[kAdjWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    AdjList& lst = Ls[w];
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const double* __restrict__ mom = a.t.mom;
    const int4* __restrict__ info = a.t.info;
    const int* __restrict__ dlf = a.t.depth_leaf;
    const double* __restrict__ X = a.x;
    const double* __restrict__ Y = a.y;
    const double* __restrict__ Z = a.z;
    const int8_t* __restrict__ SP = a.sp;

    for (int chunk = 0; true;) {
        if (lane == 0) chunk = atomicAdd(a.work, 1);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= a.nchunks) break;
        const int4 ck = a.chunks[chunk];
        const bool valid = lane < ck.y;
        const int t = valid ? (a.targets ? a.targets[ck.x + lane] : ck.x + lane) : -1;
        const int root = a.pos_off[a.t.cloud_start ? a.t.cloud_start[ck.z] : 0];
        const int end = info[root].z;
        const double xt = valid ? X[t] : 0.0, yt = valid ? Y[t] : 0.0, zt = valid ? Z[t] : 0.0;
        double l[3] = {0.0, 0.0, 0.0};
        double qm = 0.0;
        if (valid) {
            l[0] = lam[3 * (size_t)t];
            l[1] = lam[3 * (size_t)t + 1];
            l[2] = lam[3 * (size_t)t + 2];
            const int s = SP[t];
            qm = (s ? q1 : q0) / a.msp[s];
        }
        const double wv[3] = {qm * l[0], qm * l[1], qm * l[2]};
        double mt[3] = {0.0, 0.0, 0.0};
        int skip = valid ? 0 : 0x7fffffff;
        int npl = 0;

        auto flush = [&]() {
            __syncwarp();
            for (int e = 0; e < npl; ++e) {
                const int nd = lst.leaf[e];
                const bool in = (lst.mask[e] >> lane) & 1u;
                const int4 inf = info[nd];
                for (int j = inf.x; j < inf.y; ++j) {
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    const double qj = SP[j] ? q1 : q0;
                    if (in && j != t) {
                        double r[3] = {xt - X[j], yt - Y[j], zt - Z[j]};
                        double g = rsqrt(dot3(r, r) + a.eps2);
                        double g3 = g * g * g, g5 = g3 * g * g;
                        double rl = dot3(r, l), rw = dot3(r, wv);
                        mt[0] += qm * qj * (l[0] * g3 - 3.0 * r[0] * rl * g5);
                        mt[1] += qm * qj * (l[1] * g3 - 3.0 * r[1] * rl * g5);
                        mt[2] += qm * qj * (l[2] * g3 - 3.0 * r[2] * rl * g5);
                        sx = -qj * (wv[0] * g3 - 3.0 * r[0] * rw * g5);
                        sy = -qj * (wv[1] * g3 - 3.0 * r[1] * rw * g5);
                        sz = -qj * (wv[2] * g3 - 3.0 * r[2] * rw * g5);
                    }
                    sx = wsum(sx);
                    sy = wsum(sy);
                    sz = wsum(sz);
                    if (lane == 0) {
                        atomicAdd(&mu[3 * (size_t)j], sx);
                        atomicAdd(&mu[3 * (size_t)j + 1], sy);
                        atomicAdd(&mu[3 * (size_t)j + 2], sz);
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
            double dx = __dsub_rn(xt, m[0]);
            double dy = __dsub_rn(yt, m[1]);
            double dz = __dsub_rn(zt, m[2]);
            double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                  __dmul_rn(dz, dz));
            const bool acc = active && (m[MR2] < d2);
            const bool opn = active && !acc;
            const unsigned int am = __ballot_sync(0xffffffffu, acc);
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
            if (am) {
                double src[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) src[k] = 0.0;
                if (acc) {
                    const double R[3] = {dx, dy, dz};
                    const double M = m[MM];
                    const double D[3] = {m[MD], m[MD + 1], m[MD + 2]};
                    const double Q[6] = {m[MQ], m[MQ + 1], m[MQ + 2], m[MQ + 3], m[MQ + 4], m[MQ + 5]};
                    const double g = rsqrt(d2 + a.eps2);
                    const double g2 = g * g, g3 = g2 * g, g5 = g3 * g2, g7 = g5 * g2;
                    const double Rl = dot3(R, l), RD = dot3(R, D), lD = dot3(l, D);
                    double T4l[3];
                    t4(R, l, Q, g, T4l);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        double hess = M * (3.0 * R[c] * Rl * g5 - l[c] * g3);
                        double dterm = -15.0 * R[c] * Rl * RD * g7 +
                                       3.0 * (l[c] * RD + D[c] * Rl + R[c] * lD) * g5;
                        mt[c] -= qm * (hess - dterm + 0.5 * T4l[c]);
                    }
                    const double Rw = dot3(R, wv);
                    double T4w[3];
                    t4(R, wv, Q, g, T4w);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        src[c] = 3.0 * R[c] * Rw * g5 - wv[c] * g3;   // alpha
                        src[9 + c] = 0.5 * T4w[c];                     // kappa
                    }
                    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int e = ia[k], c = ib[k];
                        src[3 + k] = -15.0 * Rw * R[e] * R[c] * g7 +
                                     3.0 * (wv[e] * R[c] + wv[c] * R[e] + (e == c ? Rw : 0.0)) * g5;
                    }
                }
#pragma unroll
                for (int k = 0; k < 12; ++k) src[k] = wsum(src[k]);
                if (lane == 0)
                    for (int k = 0; k < 12; ++k) atomicAdd(&adj[(size_t)node * 12 + k], src[k]);
            }
            node = next;
            if (npl == kAdjList) flush();
        }
        flush();
        if (valid) {
            atomicAdd(&mu[3 * (size_t)t], mt[0]);
            atomicAdd(&mu[3 * (size_t)t + 1], mt[1]);
            atomicAdd(&mu[3 * (size_t)t + 2], mt[2]);
        }
    }
}

// ---- FP32 form (FP32C contexts): the node-relative coordinates, records and
// borderline FP64 decisions of the FP32C walk; per-lane sums in FP32, the
// scatter into mu in FP64, the box accumulators in FP32.

// Warp sums of several values at once by halving exchanges: at each xor step a
// lane keeps half of its values and adds the partner's copy of that half, so 16
// values take 16 exchanges instead of 80 (4 values: 6 instead of 20), and the
// sums end up spread over the lanes.
// 16 values: lane L ends with value 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of L)
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = (lane & 16) != 0;
        const float keep = hi ? v[i + 8] : v[i], send = hi ? v[i] : v[i + 8];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = (lane & 8) != 0;
        const float keep = hi ? v[i + 4] : v[i], send = hi ? v[i] : v[i + 4];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = (lane & 4) != 0;
        const float keep = hi ? v[i + 2] : v[i], send = hi ? v[i] : v[i + 2];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = (lane & 2) != 0;
        const float keep = hi ? v[1] : v[0], send = hi ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// 4 values: lane L ends with value 2 b4 + b3
__device__ __forceinline__ float warp_sum4(float (&v)[4], int lane)
{
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = (lane & 16) != 0;
        const float keep = hi ? v[i + 2] : v[i], send = hi ? v[i] : v[i + 2];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    {
        const bool hi = (lane & 8) != 0;
        const float keep = hi ? v[1] : v[0], send = hi ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float r = v[0];
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

__device__ __forceinline__ float dot3f(const float* a, const float* b)
{
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

__device__ __forceinline__ void qmulf(const float* Q, const float* v, float* o)
{
    o[0] = fmaf(Q[0], v[0], fmaf(Q[1], v[1], Q[2] * v[2]));
    o[1] = fmaf(Q[1], v[0], fmaf(Q[3], v[1], Q[4] * v[2]));
    o[2] = fmaf(Q[2], v[0], fmaf(Q[4], v[1], Q[5] * v[2]));
}

// The fourth-derivative term of the expansion contracted with a vector v:
//   o_a = 105 R_a (R.v)(R.Q.R) g^9 - 15 g^7 (v_a R.Q.R + 2 (R.v)(QR)_a + 2 R_a v.QR
//         + R_a (R.v) tr Q) + 3 g^5 (v_a tr Q + 2 (Qv)_a),
// collected as coefficients of R_a, (QR)_a, v_a and (Qv)_a.  It is linear in v:
// the source side's weight w = (q/m) lambda takes it as q/m times lambda's.
__device__ __forceinline__ void t4f(const float* R, const float* v, const float* Q, float g5,
                                    float g7, float g9, float Rv, float* o)
{
    float QR[3], Qv[3];
    qmulf(Q, R, QR);
    qmulf(Q, v, Qv);
    const float RQR = dot3f(R, QR), trQ = Q[0] + Q[3] + Q[5];
    const float cv = 3.f * g5 * trQ - 15.f * g7 * RQR;
    const float cqv = 6.f * g5;
    const float vQR = dot3f(v, QR);
    const float cr = 105.f * Rv * RQR * g9 - 15.f * g7 * (2.f * vQR + Rv * trQ);
    const float cq = -30.f * g7 * Rv;
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = fmaf(cr, R[a], fmaf(cq, QR[a], fmaf(cv, v[a], cqv * Qv[a])));
}

// 8 blocks of 128 per SM (64 registers): more resident warps for this issue-bound
// walk than the compiler's own choice, without spills
__global__ void __launch_bounds__(kAdjThreads, 8)
k_walk_adjoint_f32(WalkArgs a, const double* __restrict__ lam, double* __restrict__ mu,
                   float* __restrict__ adj)
{
    __shared__ AdjList Ls[kAdjWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    AdjList& lst = Ls[w];
    const double q0 = a.qsp[0], q1 = a.qsp[1];
    const float4* __restrict__ F = a.t.f32;
    const float4* __restrict__ S = a.src32;
    const float eps2 = (float)a.eps2;

    for (int chunk = 0; true;) {
        if (lane == 0) chunk = atomicAdd(a.work, 1);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= a.nchunks) break;
        const int4 ck = a.chunks[chunk];
        const bool valid = lane < ck.y;
        const int t = valid ? (a.targets ? a.targets[ck.x + lane] : ck.x + lane) : -1;
        const int root = a.pos_off[a.t.cloud_start ? a.t.cloud_start[ck.z] : 0];
        const int end = __float_as_int(F[(size_t)root * kF32 + 1].w);
        float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f;
        float l[3] = {0.f, 0.f, 0.f};
        float qm = 0.f;
        if (valid) {
            // relative to the centre of the cloud's cube, as the box records are
            const double* cc = a.cubes[ck.z].c;
            double X = a.x[t] - cc[0], Y = a.y[t] - cc[1], Z = a.z[t] - cc[2];
            xh = (float)X; yh = (float)Y; zh = (float)Z;
            xl = (float)(X - (double)xh); yl = (float)(Y - (double)yh); zl = (float)(Z - (double)zh);
            l[0] = (float)lam[3 * (size_t)t];
            l[1] = (float)lam[3 * (size_t)t + 1];
            l[2] = (float)lam[3 * (size_t)t + 2];
            const int s = a.sp[t];
            qm = (float)((s ? q1 : q0) / a.msp[s]);
        }
        // the source side's weight is w = (q/m) lambda: every source-side term is
        // q/m times the target side's form in lambda
        float mt[3] = {0.f, 0.f, 0.f};
        int skip = valid ? 0 : 0x7fffffff;
        int npl = 0;

        auto flush = [&]() {
            __syncwarp();
            for (int e = 0; e < npl; ++e) {
                const int nd = lst.leaf[e];
                const bool in = (lst.mask[e] >> lane) & 1u;
                const float4* r = F + (size_t)nd * kF32;
                const float4 A = r[0], B = r[1], C = r[2];
                const float rx = (xh + A.x) + (xl + B.x), ry = (yh + A.y) + (yl + B.y),
                            rz = (zh + A.z) + (zl + B.z);
                const int jb = __ldg(&a.t.info[nd].x), je = __float_as_int(C.y);
                for (int j = jb; j < je; ++j) {
                    const float4 P = __ldg(S + (j & ~1)), Q = __ldg(S + (j & ~1) + 1);
                    const bool odd = j & 1;
                    float sx = 0.f, sy = 0.f, sz = 0.f;
                    const float qj = odd ? Q.w : Q.z;
                    if (in && j != t) {
                        float r3[3] = {rx + (odd ? P.y : P.x), ry + (odd ? P.w : P.z),
                                       rz + (odd ? Q.y : Q.x)};
                        float g = rsqrt_ftz(dot3f(r3, r3) + eps2);
                        float g3 = g * g * g, g5 = g3 * g * g;
                        const float rl = dot3f(r3, l), qq = qm * qj;
                        // the pair's term on the target; the source takes its negative
                        const float cl = qq * g3, cr = -3.f * qq * rl * g5;
                        float tv[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            tv[c] = fmaf(cl, l[c], cr * r3[c]);
                            mt[c] += tv[c];
                        }
                        sx = -tv[0];
                        sy = -tv[1];
                        sz = -tv[2];
                    }
                    float sv[4] = {sx, sy, sz, 0.f};
                    const float tot = warp_sum4(sv, lane);
                    const int comp = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
                    if ((lane & 7) == 0 && comp < 3)
                        atomicAdd(&mu[3 * (size_t)j + comp], (double)tot);
                }
            }
            npl = 0;
            __syncwarp();
        };

        int node = root;
        while (node < end) {
            const float4* r = F + (size_t)node * kF32;
            const float4 A = r[0], B = r[1], C = r[2];
            const int nxt = __float_as_int(B.w);
            const bool leaf = __float_as_int(C.y) >= 0;
            const bool active = node >= skip;
            const float R[3] = {(xh + A.x) + (xl + B.x), (yh + A.y) + (yl + B.y),
                                (zh + A.z) + (zl + B.z)};
            const float d2 = dot3f(R, R);
            bool acc = active && (A.w < d2);
            if (active && fabsf(d2 - A.w) <= 4e-6f * d2) {
                const double* m = a.t.mom + (size_t)node * kMom;
                double dx = __dsub_rn(a.x[t], m[0]), dy = __dsub_rn(a.y[t], m[1]),
                       dz = __dsub_rn(a.z[t], m[2]);
                acc = m[MR2] < __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                         __dmul_rn(dz, dz));
            }
            const bool opn = active && !acc;
            const unsigned int am = __ballot_sync(0xffffffffu, acc);
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
            if (am) {
                float src[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) src[k] = 0.f;
                if (acc) {
                    const float4 D4 = r[3], E4 = r[4];
                    const float M = C.z;
                    const float D[3] = {C.w, D4.x, D4.y};
                    const float Q[6] = {D4.z, D4.w, E4.x, E4.y, E4.z, E4.w};
                    const float g = rsqrt_ftz(d2 + eps2);
                    const float g2 = g * g, g3 = g2 * g, g5 = g3 * g2, g7 = g5 * g2, g9 = g7 * g2;
                    const float Rl = dot3f(R, l), RD = dot3f(R, D), lD = dot3f(l, D);
                    float T4l[3];
                    t4f(R, l, Q, g5, g7, g9, Rl, T4l);
                    // monopole Hessian M (3 R (R.l) g^5 - l g^3) minus the dipole term
                    // -15 R (R.l)(R.D) g^7 + 3 (l (R.D) + D (R.l) + R (l.D)) g^5,
                    // collected as coefficients of R, l and D
                    const float aR = 3.f * g5 * (M * Rl - lD) + 15.f * g7 * Rl * RD;
                    const float al = -(M * g3 + 3.f * g5 * RD);
                    const float aD = -3.f * g5 * Rl;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        mt[c] -= qm * fmaf(aR, R[c], fmaf(al, l[c], fmaf(aD, D[c], 0.5f * T4l[c])));
                    // source side in w = (q/m) lambda: q/m times the lambda forms
                    const float Rw = qm * Rl, w5 = 3.f * qm * g5, w3 = qm * g3, hq = 0.5f * qm;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        src[c] = fmaf(3.f * Rw * g5, R[c], -w3 * l[c]);
                        src[9 + c] = hq * T4l[c];
                    }
                    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
                    const float r7 = -15.f * Rw * g7;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int e = ia[k], c = ib[k];
                        src[3 + k] = fmaf(r7 * R[e], R[c],
                                          w5 * (l[e] * R[c] + l[c] * R[e] + (e == c ? Rl : 0.f)));
                    }
                }
                float sv[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) sv[k] = k < 12 ? src[k] : 0.f;
                const float tot = warp_sum16(sv, lane);
                const int term = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 +
                                 ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                if ((lane & 1) == 0 && term < 12) atomicAdd(&adj[(size_t)node * 12 + term], tot);
            }
            node = next;
            if (npl == kAdjList) flush();
        }
        flush();
        if (valid) {
            atomicAdd(&mu[3 * (size_t)t], (double)mt[0]);
            atomicAdd(&mu[3 * (size_t)t + 1], (double)mt[1]);
            atomicAdd(&mu[3 * (size_t)t + 2], (double)mt[2]);
        }
    }
}

// Every particle of a leaf receives the source-side terms of the leaf and of
// all its ancestors: q_s (sum alpha - sum Gamma (x_s - c)) + |q_s| sum kappa / S0.
template <class TA>
__global__ void k_adjoint_push(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, const int8_t* __restrict__ sp,
                               const double* __restrict__ qsp, Tree t,
                               const TA* __restrict__ adj, double* __restrict__ mu)
{
    const int nl = t.count[kMaxDepth + 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
        const int leaf = t.leaf_list[i];
        double A[3] = {0, 0, 0}, G[6] = {0, 0, 0, 0, 0, 0}, Cc[3] = {0, 0, 0}, K[3] = {0, 0, 0};
        for (int nd = leaf; nd >= 0; nd = t.info[nd].w) {
            double r[12];
            for (int k = 0; k < 12; ++k) r[k] = (double)adj[(size_t)nd * 12 + k];
            const double* m = t.mom + (size_t)nd * kMom;
            double c[3] = {m[MC], m[MC + 1], m[MC + 2]};
            double Gc[3];
            qmul(r + 3, c, Gc);
            const double inv = m[MS0] > 0.0 ? 1.0 / m[MS0] : 0.0;
            for (int k = 0; k < 3; ++k) {
                A[k] += r[k];
                Cc[k] += Gc[k];
                K[k] += r[9 + k] * inv;
            }
            for (int k = 0; k < 6; ++k) G[k] += r[3 + k];
        }
        const int4 inf = t.info[leaf];
        for (int s = inf.x; s < inf.y; ++s) {
            const double qs = sp[s] ? qsp[1] : qsp[0];
            const double xs[3] = {x[s], y[s], z[s]};
            double Gx[3];
            qmul(G, xs, Gx);
            for (int k = 0; k < 3; ++k)
                mu[3 * (size_t)s + k] += qs * (A[k] - Gx[k] + Cc[k]) + fabs(qs) * K[k];
        }
    }
}

template <class TA>
__global__ void k_zero_adj(const int* __restrict__ nnodes, TA* __restrict__ adj)
{
    const size_t total = (size_t)*nnodes * 12;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        adj[i] = (TA)0;
}

// dst[t] = src[id[t]] for N x 3 arrays (caller order -> key order)
__global__ void k_gather3(const double* __restrict__ src, const unsigned int* __restrict__ id, int n,
                          double* __restrict__ dst)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    size_t j = id[t];
    dst[3 * (size_t)t] = src[3 * j];
    dst[3 * (size_t)t + 1] = src[3 * j + 1];
    dst[3 * (size_t)t + 2] = src[3 * j + 2];
}

// dst[id[t]] += src[t] for N x 3 arrays (key order -> caller order)
__global__ void k_scatter_add3(const double* __restrict__ src, const unsigned int* __restrict__ id,
                               int n, double* __restrict__ dst)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    size_t j = id[t];
    dst[3 * j] += src[3 * (size_t)t];
    dst[3 * j + 1] += src[3 * (size_t)t + 1];
    dst[3 * j + 2] += src[3 * (size_t)t + 2];
}

// out = coefficient(species) * lam_v: electrons ce, ions ci
__global__ void k_kick_lambda(const double* __restrict__ lam_v, const int8_t* __restrict__ sp, int n,
                              double ce, double ci, double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f = sp[i] ? ce : ci;
    for (int k = 0; k < 3; ++k) out[3 * (size_t)i + k] = f * lam_v[3 * (size_t)i + k];
}

// y += a x over n x 3
__global__ void k_axpy3(double* __restrict__ y, const double* __restrict__ x, double a, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    y[i] += a * x[i];
}

// lam_v = m_e v on electrons, 0 on ions; loss = sum 1/2 m_e v^2 (deterministic: one block)
__global__ void k_ke_seed(const double* __restrict__ v, const int8_t* __restrict__ sp, int n,
                          double me, double* __restrict__ lam_v, double* __restrict__ loss)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bool e = sp[i] != 0;
        for (int k = 0; k < 3; ++k) {
            double vv = v[3 * (size_t)i + k];
            lam_v[3 * (size_t)i + k] = e ? me * vv : 0.0;
            if (e) acc += 0.5 * me * vv * vv;
        }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sh[0];
}

}  // namespace

void launch_gather3(const double* src, const unsigned int* id, int n, double* dst, cudaStream_t s)
{
    count_launch(1);
    k_gather3<<<(n + 255) / 256, 256, 0, s>>>(src, id, n, dst);
}

void launch_scatter_add3(const double* src, const unsigned int* id, int n, double* dst,
                         cudaStream_t s)
{
    count_launch(1);
    k_scatter_add3<<<(n + 255) / 256, 256, 0, s>>>(src, id, n, dst);
}

void launch_kick_lambda(const double* lam_v, const int8_t* sp, int n, double ce, double ci,
                        double* out, cudaStream_t s)
{
    count_launch(1);
    k_kick_lambda<<<(n + 255) / 256, 256, 0, s>>>(lam_v, sp, n, ce, ci, out);
}

void launch_axpy3(double* y, const double* x, double a, int n, cudaStream_t s)
{
    count_launch(1);
    k_axpy3<<<(3 * n + 255) / 256, 256, 0, s>>>(y, x, a, n);
}

void launch_ke_seed(const double* v, const int8_t* sp, int n, double me, double* lam_v,
                    double* loss, cudaStream_t s)
{
    count_launch(1);
    k_ke_seed<<<1, 256, 0, s>>>(v, sp, n, me, lam_v, loss);
}

void launch_walk_adjoint(const WalkArgs& a, const double* lam, double* mu, double* adj, int n,
                         int nsm, cudaStream_t s)
{
    count_launch(3);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    cudaMemsetAsync(mu, 0, sizeof(double) * 3 * (size_t)n, s);
    int blocks = nsm * 8;
    int need = (a.nchunks + kAdjWarps - 1) / kAdjWarps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (a.src32) {
        // FP32C context: FP32 walk, FP32 box accumulators (in the same buffer)
        float* adjf = reinterpret_cast<float*>(adj);
        k_zero_adj<float><<<2 * 152, 256, 0, s>>>(a.t.nnodes, adjf);
        k_walk_adjoint_f32<<<blocks, kAdjThreads, 0, s>>>(a, lam, mu, adjf);
        k_adjoint_push<float><<<4 * 152, 256, 0, s>>>(a.x, a.y, a.z, a.sp, a.qsp, a.t, adjf, mu);
    } else {
        k_zero_adj<double><<<2 * 152, 256, 0, s>>>(a.t.nnodes, adj);
        k_walk_adjoint<<<blocks, kAdjThreads, 0, s>>>(a, lam, mu, adj);
        k_adjoint_push<double><<<4 * 152, 256, 0, s>>>(a.x, a.y, a.z, a.sp, a.qsp, a.t, adj, mu);
    }
}

}  // namespace ucp
