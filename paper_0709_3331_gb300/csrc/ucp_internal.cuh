// ucp_internal.cuh -- device data layout and kernel entry points shared by the
// translation units of libucp (TREE method of arXiv 0709.3331, Sec. 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace ucp {

constexpr int kMaxDepth = 21;        // 21 bits per axis, 63-bit keys
constexpr int kWarp = 32;

// Order-preserving integer image of a double (larger double, larger image; -0 below
// +0; a NaN with the sign bit clear above every number, with it set below), so
// min/max reductions are exact, order-independent integer operations.
__device__ __forceinline__ unsigned long long ord64(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long u)
{
    return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

// Approximate reciprocal square root of the special-function unit (the
// approximation rsqrtf uses) with subnormal inputs and outputs flushed to zero,
// which spares the subnormal handling around it.  The walks call it on r^2 + eps^2
// or on |x_t - c|^2 + eps^2: below 2^-126 only for particles closer than 1e-19, whose
// FP32 field overflows in any case; for every normal input the result is rsqrtf's.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kernels launched by this process (read by ucp_stats).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

// One FP64 box record, 16 doubles (128 B), read by the FP64 walk.
// {c.x, c.y, c.z, rcrit2, M, D.x, D.y, D.z, Qxx, Qxy, Qxz, Qyy, Qyz, Qzz, S0, delta}
// rcrit2 = (s/theta + delta)^2 is filled per walk (it depends on theta).
constexpr int kMom = 16;
enum MomIdx { MC = 0, MR2 = 3, MM = 4, MD = 5, MQ = 8, MS0 = 14, MDELTA = 15 };

// One FP32C box record, 5 float4 (80 B):
//   A = {-ch.x, -ch.y, -ch.z, rcrit2}   ch = fp32(c), cl = fp32(c - ch)
//   B = {-cl.x, -cl.y, -cl.z, bits(next)}
//   C = {-tr(Q)/2, bits(end or -1 for a twig), M, D.x}
//   D = {D.y, D.z, Qxx, Qxy}
//   E = {Qxz, Qyy, Qyz, Qzz}
constexpr int kF32 = 5;

// Box topology {begin, end, next, parent}; depth and leaf flag separately.
struct Tree {
    int cap;                 // box capacity
    int* nnodes;             // device scalar
    int* maxdepth;           // device scalar
    int4* info;              // {begin, end, next, parent}
    int* depth_leaf;         // depth | leaf << 8
    unsigned long long* cell;// key prefix of the box at its depth
    double* mom;             // kMom doubles per box
    float4* f32;             // kF32 float4 per box
    float* mom32;            // FP32C contexts: 16 floats per box {e xyz, S0, M, D, Q, 0, 0}
    int* child8;             // 8 child slots per box (octant order), -1 = empty
    int* arrive;             // finished children per box (moments' bottom-up sweep)
    int* leaf_list;          // the leaves, any order
    int* twig_list;          // the twigs of depth d at twig_off[d] .. + count[d]
    int* count;              // count[d] twigs of depth d (d <= 20), count[kMaxDepth + 1] leaves
    int twig_off[kMaxDepth + 2];
    // clouds: cloud[i] = cloud of key-sorted position i, whose segment is
    // [cloud_start[c], cloud_start[c + 1]); NULL cloud = one cloud over [0, n)
    const unsigned char* cloud;
    const int* cloud_start;
};

struct Cube {                // enclosing cube: centre, side, lower corner, 2^21 / side
    double c[3];
    double L;
    double lo[3];
    double kscale;
};

// ---- build (ucp_build.cu) ----
void launch_bbox(const double* x, const double* y, const double* z, int n, double* partials,
                 int nblk, Cube* cubes, const int* cloud_start, int n_clouds, cudaStream_t s);
void launch_keys(const double* x, const double* y, const double* z, int n, const Cube* cubes,
                 const unsigned char* cloud, unsigned long long* key, unsigned int* val,
                 cudaStream_t s);
struct SortScratch {
    unsigned int* ghist;           // 8 x 256 digit counts, then 9 tile counters
    unsigned int* goff;            // 8 x 256 digit offsets
    unsigned long long* status;    // 9 passes x tiles x 256 published words
    int* err;                      // raised by a wait that gave up
    unsigned int* epoch;           // tag of the published words, advanced every build
    unsigned int* test_epoch;      // tag used by the bounded-wait self-test (1)
    unsigned long long* test_keys; // 4 tiles, for the bounded-wait self-test
    unsigned int* test_vals;
};
size_t sort_status_words(int n);
size_t sort_test_words();
// returns the buffer (0 or 1) that holds the sorted keys and permutation
int launch_sort(unsigned long long* key[2], unsigned int* val[2], int n, SortScratch sc,
                const unsigned int* ids_in, const unsigned char* cloud,
                const int* cloud_start, int n_clouds, cudaStream_t s);
int sort_selftest_timeout(SortScratch sc, cudaStream_t s);
void launch_tiefix(const unsigned long long* key, unsigned int* perm, const unsigned int* ids,
                   int n, cudaStream_t s);
void launch_topology(const unsigned long long* key, int n, int leaf_cap, int* pos_cnt,
                     int* pos_off, int* scan_part, Tree t, cudaStream_t s);
void launch_moments(const double* x, const double* y, const double* z, const int8_t* sp,
                    const double* qsp, int n, const Cube* cube, Tree t, float4* src32,
                    int want_f32, cudaStream_t s);
void launch_scan(const int* in, int* out, int n, int* partials, int* total, cudaStream_t s);
size_t scan_partials_words(int n);

// ---- walk (ucp_walk.cu) ----
struct WalkArgs {
    const double* x; const double* y; const double* z;
    const int8_t* sp;
    const double* qsp;      // charge per species (device, 2)
    const double* msp;      // mass per species (device, 2)
    const float4* src32;    // FP32C sources, pairs of particles: {nx0, nx1, ny0, ny1},
                            // {nz0, nz1, q0, q1} with n = c_leaf - x (key order)
    Tree t;
    const int* targets;     // key-order slots of the targets, or NULL = all
    int ntargets;
    const int4* chunks;     // {first target index, count <= 32, cloud, 0}, one cloud each
    int nchunks;
    const int* pos_off;     // first box started at each sorted position (the roots)
    const Cube* cubes;      // per cloud: FP32C coordinates are taken relative to the centre
    double eps2;
    int kelbg;              // electron-ion pairs use the Kelbg form (Sec. 2.1 Eq. 3)
    double lambda;          // its fixed lambda_ei
    double* ax; double* ay; double* az; double* phi;  // key order; phi may be NULL
    int* cnt_p2p; int* cnt_m2p;                        // key order
    int* work;              // dynamic work counter (zeroed before launch)
    int* err;               // raised by a bounded wait that gave up
    unsigned long long* stats; // {p2p, m2p}
};
void launch_mac_prepare(Tree t, const Cube* cube, double theta, int want_f32, cudaStream_t s);
void launch_walk_fp64(const WalkArgs& a, int nsm, cudaStream_t s);
void launch_walk_fp32c(const WalkArgs& a, int nsm, cudaStream_t s, int shape);
int walk_shape_count();
// Reorders a chunk list longest-first by the cost (20 per pair + 64 per multipole)
// its targets had in the walk just finished; cost and tmp hold nchunks entries.
void launch_chunk_order(int4* chunks, int nchunks, const int* targets, const int* cnt_p2p,
                        const int* cnt_m2p, float* cost, int4* tmp, cudaStream_t s);

// ---- adjoint (ucp_adjoint.cu) ----
// mu (n particles, key order) = (d a / d x)^T lam over the targets of a (all
// particles when a.targets is NULL; the others must have lam = 0)
void launch_walk_adjoint(const WalkArgs& a, const double* lam, double* mu, double* adj, int n,
                         int nsm, cudaStream_t s);
void launch_gather3(const double* src, const unsigned int* id, int n, double* dst, cudaStream_t s);
void launch_scatter_add3(const double* src, const unsigned int* id, int n, double* dst,
                         cudaStream_t s);
void launch_kick_lambda(const double* lam_v, const int8_t* sp, int n, double ce, double ci,
                        double* out, cudaStream_t s);
void launch_axpy3(double* y, const double* x, double a, int n, cudaStream_t s);
void launch_ke_seed(const double* v, const int8_t* sp, int n, double me, double* lam_v,
                    double* loss, cudaStream_t s);

// ---- push and reductions (ucp_push.cu) ----
void launch_permute(const unsigned int* perm, int n, const double* const* src6, double* const* dst6,
                    const int8_t* sp_in, int8_t* sp_out, const unsigned int* id_in,
                    unsigned int* id_out, cudaStream_t s);
void launch_kick(double* vx, double* vy, double* vz, const double* ax, const double* ay,
                 const double* az, const int8_t* sp, int species, double h, int n, int times,
                 cudaStream_t s);
// list[0 .. count) = the slots whose species is `species`, in slot order;
// partials holds scan_partials_words(n) ints
void launch_select(const int8_t* sp, int species, int n, int* list, int* partials, int* count,
                   cudaStream_t s);
void launch_drift(double* x, double* y, double* z, const double* vx, const double* vy,
                  const double* vz, double dt, int n, cudaStream_t s);
void launch_energy(const double* vx, const double* vy, const double* vz, const double* phi,
                   const int8_t* sp, const double* qsp, const double* msp, int n,
                   double* partials, int nblk, double* out6, cudaStream_t s);
void launch_energy_clouds(const double* vx, const double* vy, const double* vz, const double* phi,
                          const int8_t* sp, const double* qsp, const double* msp,
                          const int* cloud_start, int n_clouds, double* out, cudaStream_t s);
void launch_scatter3(const double* ax, const double* ay, const double* az, const unsigned int* id,
                     int n, double* out, cudaStream_t s);
void launch_scatter1(const double* a, const unsigned int* id, int n, double* out, cudaStream_t s);
void launch_scatter_int(const int* a, const unsigned int* id, int n, int* out, cudaStream_t s);
void launch_deinterleave(const double* aos, int n, double* x, double* y, double* z,
                         cudaStream_t s);
void launch_check_state(const double* pos, const double* vel, const int8_t* sp, int n, int* flags,
                        cudaStream_t s);
void launch_iota(unsigned int* a, int n, cudaStream_t s);

}  // namespace ucp
