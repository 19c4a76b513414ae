// ucp_runtime.cu -- the C ABI of include/ucp.h: context, device memory, and
// the order of kernels for TREE construction (Sec. 3), the particle-TREE walk
// and the split-step velocity Verlet push (Sec. 2) of arXiv 0709.3331.
#include "ucp.h"
#include "ucp_internal.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

using namespace ucp;

std::atomic<unsigned long long> ucp::g_launches{0};

struct ucp_ctx {
    int n = 0, leaf_cap = 1, precision = UCP_FP64;
    int potential = UCP_POT_PLUMMER;
    double lambda_ei = 1.0;
    double q[2] = {1, -1}, m[2] = {1, 1};
    cudaStream_t s = nullptr;
    int nsm = 152;
    int device = 0;

    // particle state in key order, two buffer sets (permutation ping-pong)
    double* st[2][6] = {};   // x y z vx vy vz
    int8_t* sp[2] = {};
    unsigned int* id[2] = {};
    int cur = 0;
    double *ax = nullptr, *ay = nullptr, *az = nullptr, *phi = nullptr;

    unsigned long long* key[2] = {};
    unsigned int* val[2] = {};
    SortScratch sort = {};
    int* scan_part = nullptr;
    int* pos_cnt = nullptr;
    int* pos_off = nullptr;
    Tree t = {};
    float4* src32 = nullptr;
    Cube* cube = nullptr;
    double* bbox_part = nullptr;
    int bbox_nblk = 1;
    double* qsp = nullptr;
    double* msp = nullptr;
    int* tlist = nullptr;    // selected targets (electrons), key order
    int* tcount = nullptr;
    int* cnt_p2p = nullptr;
    int* cnt_m2p = nullptr;
    int* work = nullptr;
    unsigned long long* stats = nullptr;  // {p2p, m2p}
    double* en_part = nullptr;
    int en_nblk = 1;
    double* en_out = nullptr;
    int* flags = nullptr;
    double* stage = nullptr;  // n x 6 doubles for host transfers and layout changes
    int8_t* stage_sp = nullptr;
    int8_t* sp_caller = nullptr;  // species in caller order
    int* stage_int = nullptr;

    int n_e = 0;
    // clouds: independent particle sets in fixed segments of every order
    int n_clouds = 1;
    std::vector<int> cloud_start_h;    // n_clouds + 1
    int* cloud_start = nullptr;        // device copy
    unsigned char* cloud = nullptr;    // cloud of each slot (batches only)
    int4* chunks_all = nullptr;        // walk chunks over all particles
    int4* chunks_e = nullptr;          // walk chunks over the compacted electrons
    float* chunk_cost = nullptr;       // per chunk, for the longest-first order
    int4* chunk_tmp = nullptr;
    int n_chunks_all = 0, n_chunks_e = 0, n_chunks_all_cap = 0;
    int sorted_buf = 0;                // key[] / val[] buffer of the last sort
    std::vector<double> cloud_energy;  // per-cloud {KE_i, KE_e, PE, px, py, pz} of the last energy
    bool have_state = false, tree_valid = false, acc_valid = false;
    bool phi_valid = false;           // phi of every particle at the current positions
    double phi_theta = -1.0, phi_eps = -1.0;
    int64_t steps = 0, walk_targets = 0, walk_launches = 0;
    unsigned long long launch_base = 0;

    // captured blocks of the split-step push (ucp_set_graphs)
    struct GraphEntry {
        int kk, cur_in, cur_out;
        int n_e, n_chunks_all, n_chunks_e;  // launch parameters a new state can change
        double dt_e, theta, eps;
        bool prof;                          // walks bracketed by event-record nodes
        cudaGraph_t graph;                  // kept while exec lives (its nodes are re-pointed)
        cudaGraphExec_t exec;
        unsigned long long launches;
        std::vector<cudaGraphNode_t> ev_nodes;  // {begin, end} per walk, in walk order
    };
    bool use_graphs = false;
    int walk_shape = 0;                // launch shape of the FP32C walk (ucp_autotune)
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;

    bool prof = false;
    // while a profiled block is captured: placeholder events, recorded as graph nodes
    bool cap_prof = false;
    std::vector<cudaEvent_t> cap_ev;
    size_t cap_ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;

    std::string err;
    std::vector<void*> allocs;
};

namespace {

int fail(ucp_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(c, UCP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int check_launch(ucp_ctx* c, const char* where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, UCP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return UCP_OK;
}

template <class T>
int dalloc(ucp_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, UCP_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = (T*)q;
    return UCP_OK;
}

// Upper bound on the number of boxes: depth d holds at most 8^d boxes, at most
// n, and at most 8 per twig of depth d-1, of which there are <= n/(leaf_cap+1).
int64_t box_capacity(int64_t n, int leaf_cap)
{
    int64_t twigs = n / (leaf_cap + 1);
    int64_t total = 0, pow8 = 1;
    for (int d = 0; d <= kMaxDepth; ++d) {
        int64_t lim = n;
        if (d > 0 && 8 * twigs < lim) lim = 8 * twigs;
        if (pow8 < lim) lim = pow8;
        total += lim;
        if (pow8 < ((int64_t)1 << 40)) pow8 *= 8;
    }
    return total < 1 ? 1 : total;
}

// the next placeholder event of a capture (event-record node in the graph)
static void cap_record(ucp_ctx* c)
{
    if (c->cap_ev_used == c->cap_ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->cap_ev.push_back(e);
    }
    cudaEventRecordWithFlags(c->cap_ev[c->cap_ev_used++], c->s, cudaEventRecordExternal);
}

void prof_begin(ucp_ctx* c)
{
    if (!c->prof) return;
    if (c->cap_prof) {
        cap_record(c);
        return;
    }
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        c->ev.push_back({a, b});
    }
    cudaEventRecord(c->ev[c->ev_used].first, c->s);
}

void prof_end(ucp_ctx* c)
{
    if (!c->prof) return;
    if (c->cap_prof) {
        cap_record(c);
        return;
    }
    cudaEventRecord(c->ev[c->ev_used].second, c->s);
    ++c->ev_used;
}

// Sec. 3 construction: cube, keys, sort, permutation of the state, boxes, moments.
int build(ucp_ctx* c)
{
    int n = c->n, k = c->cur;
    const int* cs = c->n_clouds > 1 ? c->cloud_start : nullptr;
    launch_bbox(c->st[k][0], c->st[k][1], c->st[k][2], n, c->bbox_part, c->bbox_nblk, c->cube,
                cs, c->n_clouds, c->s);
    launch_keys(c->st[k][0], c->st[k][1], c->st[k][2], n, c->cube, c->t.cloud, c->key[0],
                c->val[0], c->s);
    const int b = launch_sort(c->key, c->val, n, c->sort, c->id[k], c->t.cloud, c->cloud_start,
                              c->n_clouds, c->s);
    c->sorted_buf = b;
    const double* src[6];
    double* dst[6];
    for (int a = 0; a < 6; ++a) {
        src[a] = c->st[k][a];
        dst[a] = c->st[k ^ 1][a];
    }
    launch_permute(c->val[b], n, src, dst, c->sp[k], c->sp[k ^ 1], c->id[k], c->id[k ^ 1], c->s);
    c->cur = k ^ 1;
    k = c->cur;
    launch_topology(c->key[b], n, c->leaf_cap, c->pos_cnt, c->pos_off, c->scan_part, c->t, c->s);
    launch_moments(c->st[k][0], c->st[k][1], c->st[k][2], c->sp[k], c->qsp, n, c->cube, c->t,
                   c->src32, c->precision == UCP_FP32C, c->s);
    c->tree_valid = true;
    c->acc_valid = false;
    c->phi_valid = false;
    return check_launch(c, "tree build");
}

// One walk over all particles (electrons_only = 0) or the electrons.
int force(ucp_ctx* c, double theta, double eps, int electrons_only, bool want_phi)
{
    int k = c->cur;
    int f32 = c->precision == UCP_FP32C;
    launch_mac_prepare(c->t, c->cube, theta, f32, c->s);
    WalkArgs a;
    a.x = c->st[k][0];
    a.y = c->st[k][1];
    a.z = c->st[k][2];
    a.sp = c->sp[k];
    a.qsp = c->qsp;
    a.msp = c->msp;
    a.src32 = c->src32;
    a.t = c->t;
    if (electrons_only) {
        launch_select(c->sp[k], UCP_ELECTRON, c->n, c->tlist, c->scan_part, c->tcount, c->s);
        a.targets = c->tlist;
        a.ntargets = c->n_e;
        a.chunks = c->chunks_e;
        a.nchunks = c->n_chunks_e;
    } else {
        a.targets = nullptr;
        a.ntargets = c->n;
        a.chunks = c->chunks_all;
        a.nchunks = c->n_chunks_all;
    }
    a.pos_off = c->pos_off;
    a.cubes = c->cube;
    a.eps2 = eps * eps;
    a.kelbg = c->potential == UCP_POT_KELBG;
    a.lambda = c->lambda_ei;
    a.ax = c->ax;
    a.ay = c->ay;
    a.az = c->az;
    a.phi = want_phi ? c->phi : nullptr;
    a.cnt_p2p = c->cnt_p2p;
    a.cnt_m2p = c->cnt_m2p;
    a.work = c->work;
    a.err = c->sort.err;
    a.stats = c->stats;
    cudaMemsetAsync(c->cnt_p2p, 0, sizeof(int) * (size_t)c->n, c->s);
    cudaMemsetAsync(c->cnt_m2p, 0, sizeof(int) * (size_t)c->n, c->s);
    if (a.ntargets > 0) {
        prof_begin(c);
        if (f32) launch_walk_fp32c(a, c->nsm, c->s, c->walk_shape);
        else launch_walk_fp64(a, c->nsm, c->s);
        prof_end(c);
        // the next walk over the same targets takes its chunks longest-first
        launch_chunk_order(electrons_only ? c->chunks_e : c->chunks_all, a.nchunks, a.targets,
                           c->cnt_p2p, c->cnt_m2p, c->chunk_cost, c->chunk_tmp, c->s);
        c->walk_targets += a.ntargets;
        c->walk_launches += 1;
    }
    if (!electrons_only) c->acc_valid = true;
    if (!electrons_only && want_phi) {
        c->phi_valid = true;
        c->phi_theta = theta;
        c->phi_eps = eps;
    }
    return check_launch(c, "tree walk");
}

// Walk chunks: up to 32 consecutive targets of one cloud.  All-particle chunks
// cover each cloud's segment; electron chunks cover each cloud's run in the
// compacted electron list (electrons keep their cloud order under sorting).
// Targets per walk chunk: 32 (one per lane).  An FP64 context too small to give
// every SM two chunks takes narrower chunks (down to 8 targets), so more warps
// share the latency-bound FP64 walk; its sums do not depend on which targets
// share a warp, so the results are the same.  The FP32C walk's batched sums do
// depend on the warp's company, so it keeps 32.
static int chunk_width(ucp_ctx* c)
{
    if (c->precision != UCP_FP64) return 32;
    int w = 32;
    while (w > 8) {
        int64_t nch = 0;
        for (int cl = 0; cl < c->n_clouds; ++cl)
            nch += (c->cloud_start_h[cl + 1] - c->cloud_start_h[cl] + w - 1) / w;
        if (nch >= 2 * (int64_t)c->nsm) break;
        w /= 2;
    }
    return w;
}

int build_chunks(ucp_ctx* c, const std::vector<int>& ne_per_cloud)
{
    std::vector<int4> all, el;
    int e0 = 0;
    const int W = chunk_width(c);
    for (int cl = 0; cl < c->n_clouds; ++cl) {
        int b = c->cloud_start_h[cl], e = c->cloud_start_h[cl + 1];
        for (int t = b; t < e; t += W) all.push_back(make_int4(t, std::min(W, e - t), cl, 0));
        int ne = ne_per_cloud[cl];
        for (int t = 0; t < ne; t += W) el.push_back(make_int4(e0 + t, std::min(W, ne - t), cl, 0));
        e0 += ne;
    }
    if ((int)all.size() > c->n_chunks_all_cap || (int)el.size() > c->n_chunks_all_cap)
        return fail(c, UCP_EINVAL, "internal: chunk capacity");
    c->n_chunks_all = (int)all.size();
    c->n_chunks_e = (int)el.size();
    CK(cudaMemcpyAsync(c->chunks_all, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice,
                       c->s));
    if (!el.empty())
        CK(cudaMemcpyAsync(c->chunks_e, el.data(), sizeof(int4) * el.size(),
                           cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    return UCP_OK;
}

// A bounded device-side wait that gave up leaves a flag; calls that synchronise
// report it (the flag stays raised until the next ucp_set_state).
int device_error(ucp_ctx* c)
{
    int e = 0;
    if (cudaMemcpy(&e, c->sort.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, UCP_ECUDA, "reading the device error flag failed");
    if (e) return fail(c, UCP_ETIMEOUT, "a bounded device-side wait gave up");
    return UCP_OK;
}

int valid_walk_args(ucp_ctx* c, double theta, double eps)
{
    if (!(theta >= 0.0 && theta <= 1.0)) return fail(c, UCP_EINVAL, "theta must be in [0, 1]");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(c, UCP_EINVAL, "eps must be >= 0");
    return UCP_OK;
}

}  // namespace

extern "C" {

const char* ucp_strerror(int code)
{
    switch (code) {
    case UCP_OK: return "ok";
    case UCP_EINVAL: return "invalid argument";
    case UCP_ENOMEM: return "out of memory";
    case UCP_ECUDA: return "CUDA error";
    case UCP_ENONFINITE: return "non-finite position or velocity";
    case UCP_ETIMEOUT: return "device wait timed out";
    case UCP_ESTATE: return "no particle state set";
    default: return "unknown error";
    }
}

const char* ucp_last_error(ucp_ctx* c) { return c ? c->err.c_str() : "null context"; }

void ucp_destroy(ucp_ctx* c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    else cudaDeviceSynchronize();
    for (void* p : c->allocs) cudaFree(p);
    for (auto& e : c->ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (auto& g : c->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    for (cudaEvent_t e : c->cap_ev) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

int ucp_create(ucp_ctx** out, const ucp_params* p)
{
    if (!out || !p) return UCP_EINVAL;
    *out = nullptr;
    const int64_t n = p->n;
    return ucp_create_batch(out, p, 1, &n);
}

int ucp_create_batch(ucp_ctx** out, const ucp_params* p, int32_t n_clouds, const int64_t* sizes)
{
    if (!out || !p || !sizes) return UCP_EINVAL;
    *out = nullptr;
    if (n_clouds < 1 || n_clouds > UCP_MAX_CLOUDS) return UCP_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < n_clouds; ++i) {
        if (sizes[i] < 1) return UCP_EINVAL;
        total += sizes[i];
    }
    if (total > 0x7fffffffLL) return UCP_EINVAL;
    if (n_clouds > 1 && p->n != 0 && p->n != total) return UCP_EINVAL;
    if (p->leaf_cap < 1 || p->leaf_cap > 1024) return UCP_EINVAL;
    if (p->precision != UCP_FP64 && p->precision != UCP_FP32C) return UCP_EINVAL;
    for (int s = 0; s < 2; ++s)
        if (!(p->m[s] > 0.0) || !std::isfinite(p->m[s]) || !std::isfinite(p->q[s]))
            return UCP_EINVAL;
    if (p->potential != UCP_POT_PLUMMER && p->potential != UCP_POT_KELBG) return UCP_EINVAL;
    if (p->potential == UCP_POT_KELBG &&
        (!(p->lambda_ei > 0.0) || !std::isfinite(p->lambda_ei) || p->q[0] == p->q[1]))
        return UCP_EINVAL;
    int64_t cap = 0;
    for (int i = 0; i < n_clouds; ++i) cap += box_capacity(sizes[i], p->leaf_cap);
    if (cap > 0x7ffffff0LL) return UCP_EINVAL;

    ucp_ctx* c = new (std::nothrow) ucp_ctx();
    if (!c) return UCP_ENOMEM;
    c->n = (int)total;
    c->n_clouds = n_clouds;
    c->cloud_start_h.assign(n_clouds + 1, 0);
    for (int i = 0; i < n_clouds; ++i) c->cloud_start_h[i + 1] = c->cloud_start_h[i] + (int)sizes[i];
    c->leaf_cap = p->leaf_cap;
    c->precision = p->precision;
    c->potential = p->potential;
    c->lambda_ei = p->potential == UCP_POT_KELBG ? p->lambda_ei : 1.0;
    for (int s = 0; s < 2; ++s) {
        c->q[s] = p->q[s];
        c->m[s] = p->m[s];
    }
    c->s = (cudaStream_t)p->cuda_stream;
    int rc = UCP_OK;
    auto bail = [&](int code) {
        std::string msg = c->err;
        ucp_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(UCP_ECUDA);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    size_t n = (size_t)c->n;
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 6; ++a)
            if ((rc = dalloc(c, &c->st[b][a], n))) return bail(rc);
        if ((rc = dalloc(c, &c->sp[b], n))) return bail(rc);
        if ((rc = dalloc(c, &c->id[b], n))) return bail(rc);
        if ((rc = dalloc(c, &c->key[b], n))) return bail(rc);
        if ((rc = dalloc(c, &c->val[b], n))) return bail(rc);
    }
    if ((rc = dalloc(c, &c->ax, n)) || (rc = dalloc(c, &c->ay, n)) || (rc = dalloc(c, &c->az, n)) ||
        (rc = dalloc(c, &c->phi, n)))
        return bail(rc);
    if ((rc = dalloc(c, &c->sort.ghist, 8 * 256 + 9)) || (rc = dalloc(c, &c->sort.goff, 8 * 256)) ||
        (rc = dalloc(c, &c->sort.status, sort_status_words(c->n))) ||
        (rc = dalloc(c, &c->sort.err, 1)) || (rc = dalloc(c, &c->sort.epoch, 1)) ||
        (rc = dalloc(c, &c->sort.test_epoch, 1)) ||
        (rc = dalloc(c, &c->sort.test_keys, sort_test_words())) ||
        (rc = dalloc(c, &c->sort.test_vals, sort_test_words())))
        return bail(rc);
    if (cudaMemsetAsync(c->sort.status, 0, 8 * sort_status_words(c->n), c->s) != cudaSuccess ||
        cudaMemsetAsync(c->sort.err, 0, sizeof(int), c->s) != cudaSuccess ||
        cudaMemsetAsync(c->sort.epoch, 0, sizeof(unsigned int), c->s) != cudaSuccess)
        return bail(UCP_ECUDA);
    size_t spw = scan_partials_words(c->n);
    if ((rc = dalloc(c, &c->scan_part, spw))) return bail(rc);
    if ((rc = dalloc(c, &c->pos_cnt, n)) || (rc = dalloc(c, &c->pos_off, n))) return bail(rc);
    c->t.cap = (int)cap;
    size_t cz = (size_t)cap;
    if ((rc = dalloc(c, &c->t.nnodes, 1)) || (rc = dalloc(c, &c->t.maxdepth, 1)) ||
        (rc = dalloc(c, &c->t.info, cz)) || (rc = dalloc(c, &c->t.depth_leaf, cz)) ||
        (rc = dalloc(c, &c->t.cell, cz)) || (rc = dalloc(c, &c->t.mom, cz * kMom)) ||
        (rc = dalloc(c, &c->t.child8, cz * 8)) || (rc = dalloc(c, &c->t.leaf_list, cz)) ||
        (rc = dalloc(c, &c->t.arrive, cz)) ||
        (rc = dalloc(c, &c->t.count, kMaxDepth + 2)))
        return bail(rc);
    {
        // twigs of depth d: at most min(8^d, n / (leaf_cap + 1)); none at the depth cap
        int64_t off = 0, pow8 = 1;
        for (int d = 0; d <= kMaxDepth + 1; ++d) {
            c->t.twig_off[d] = (int)off;
            if (d < kMaxDepth)
                for (int i = 0; i < n_clouds; ++i) {
                    int64_t twigs = sizes[i] / (c->leaf_cap + 1);
                    off += pow8 < twigs ? pow8 : twigs;
                }
            if (pow8 < ((int64_t)1 << 40)) pow8 *= 8;
        }
        if ((rc = dalloc(c, &c->t.twig_list, (size_t)(off > 0 ? off : 1)))) return bail(rc);
    }
    if (c->precision == UCP_FP32C) {
        // sources in pairs: 2 float4 per pair of particles (padded to an even count)
        if ((rc = dalloc(c, &c->t.f32, cz * kF32)) || (rc = dalloc(c, &c->src32, n + 1)) ||
            (rc = dalloc(c, &c->t.mom32, cz * 16)))
            return bail(rc);
        // the pad slot of an odd count is read (masked) by the pair loop: keep it finite
        if (cudaMemsetAsync(c->src32, 0, sizeof(float4) * (n + 1), c->s) != cudaSuccess)
            return bail(UCP_ECUDA);
    }
    if ((rc = dalloc(c, &c->cube, (size_t)n_clouds))) return bail(rc);
    {
        int64_t biggest = 0;
        for (int i = 0; i < n_clouds; ++i) biggest = sizes[i] > biggest ? sizes[i] : biggest;
        c->bbox_nblk = (int)((biggest + 2047) / 2048);
        int lim = n_clouds > 1 ? 16 : 4 * c->nsm;
        if (c->bbox_nblk > lim) c->bbox_nblk = lim;
        if (c->bbox_nblk < 1) c->bbox_nblk = 1;
    }
    c->en_nblk = (int)((n + 2047) / 2048);
    if (c->en_nblk > 4 * c->nsm) c->en_nblk = 4 * c->nsm;
    if (c->en_nblk < 1) c->en_nblk = 1;
    if ((rc = dalloc(c, &c->bbox_part, (size_t)n_clouds * c->bbox_nblk * 6)) ||
        (rc = dalloc(c, &c->en_part, (size_t)c->en_nblk * 6)) ||
        (rc = dalloc(c, &c->en_out, (size_t)6 * n_clouds)))
        return bail(rc);
    {
        // clouds: segment starts, the (static) cloud of every slot, walk chunk capacity
        if ((rc = dalloc(c, &c->cloud_start, (size_t)n_clouds + 1))) return bail(rc);
        if (cudaMemcpyAsync(c->cloud_start, c->cloud_start_h.data(), sizeof(int) * (n_clouds + 1),
                            cudaMemcpyHostToDevice, c->s) != cudaSuccess)
            return bail(UCP_ECUDA);
        c->t.cloud_start = c->cloud_start;
        c->t.cloud = nullptr;
        if (n_clouds > 1) {
            std::vector<unsigned char> cl(n);
            for (int i = 0; i < n_clouds; ++i)
                for (int j = c->cloud_start_h[i]; j < c->cloud_start_h[i + 1]; ++j)
                    cl[j] = (unsigned char)i;
            if ((rc = dalloc(c, &c->cloud, n))) return bail(rc);
            if (cudaMemcpyAsync(c->cloud, cl.data(), n, cudaMemcpyHostToDevice, c->s) != cudaSuccess ||
                cudaStreamSynchronize(c->s) != cudaSuccess)
                return bail(UCP_ECUDA);
            c->t.cloud = c->cloud;
        }
        int64_t nch = 0;
        for (int i = 0; i < n_clouds; ++i) nch += (sizes[i] + 7) / 8;  // chunks of >= 8
        c->n_chunks_all_cap = (int)nch;
        if ((rc = dalloc(c, &c->chunks_all, (size_t)nch)) ||
            (rc = dalloc(c, &c->chunks_e, (size_t)nch)) ||
            (rc = dalloc(c, &c->chunk_cost, (size_t)nch)) ||
            (rc = dalloc(c, &c->chunk_tmp, (size_t)nch)))
            return bail(rc);
    }
    if ((rc = dalloc(c, &c->qsp, 2)) || (rc = dalloc(c, &c->msp, 2))) return bail(rc);
    if ((rc = dalloc(c, &c->tlist, n)) || (rc = dalloc(c, &c->tcount, 1)))
        return bail(rc);
    if ((rc = dalloc(c, &c->cnt_p2p, n)) || (rc = dalloc(c, &c->cnt_m2p, n)) ||
        (rc = dalloc(c, &c->work, 1)) || (rc = dalloc(c, &c->stats, 2)) ||
        (rc = dalloc(c, &c->flags, 2)))
        return bail(rc);
    if ((rc = dalloc(c, &c->stage, 6 * n)) || (rc = dalloc(c, &c->stage_sp, n)) ||
        (rc = dalloc(c, &c->sp_caller, n)) ||
        (rc = dalloc(c, &c->stage_int, 2 * n)))
        return bail(rc);
    if (cudaMemcpyAsync(c->qsp, c->q, 2 * sizeof(double), cudaMemcpyHostToDevice, c->s) ||
        cudaMemcpyAsync(c->msp, c->m, 2 * sizeof(double), cudaMemcpyHostToDevice, c->s) ||
        cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), c->s) ||
        cudaStreamSynchronize(c->s)) {
        c->err = "initial copies failed";
        return bail(UCP_ECUDA);
    }
    *out = c;
    return UCP_OK;
}

int ucp_set_state(ucp_ctx* c, const double* pos, const double* vel, const int8_t* species,
                  int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!pos || !vel || !species) return fail(c, UCP_EINVAL, "null pointer");
    size_t n = (size_t)c->n;
    const double* dpos = pos;
    const double* dvel = vel;
    const int8_t* dsp = species;
    int k = c->cur;
    std::vector<int8_t> host_sp;
    if (!on_device) {
        int ne = 0;
        for (size_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(pos[3 * i + a]) || !std::isfinite(vel[3 * i + a]))
                    return fail(c, UCP_ENONFINITE, "non-finite position or velocity");
            if (species[i] != 0 && species[i] != 1)
                return fail(c, UCP_EINVAL, "species must be 0 (ion) or 1 (electron)");
            ne += species[i] == 1;
        }
        CK(cudaMemcpyAsync(c->stage, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->s));
        CK(cudaMemcpyAsync(c->stage + 3 * n, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice,
                           c->s));
        CK(cudaMemcpyAsync(c->sp[k], species, n, cudaMemcpyHostToDevice, c->s));
        dpos = c->stage;
        dvel = c->stage + 3 * n;
        c->n_e = ne;
    } else {
        CK(cudaMemsetAsync(c->flags, 0, 2 * sizeof(int), c->s));
        launch_check_state(pos, vel, species, c->n, c->flags, c->s);
        int fl[2] = {0, 0};
        CK(cudaMemcpyAsync(fl, c->flags, sizeof(fl), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        if (fl[0]) return fail(c, UCP_ENONFINITE, "non-finite position or velocity");
        if (fl[1]) return fail(c, UCP_EINVAL, "species must be 0 (ion) or 1 (electron)");
        CK(cudaMemcpyAsync(c->sp[k], dsp, n, cudaMemcpyDeviceToDevice, c->s));
        host_sp.resize(n);
        CK(cudaMemcpyAsync(host_sp.data(), dsp, n, cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        species = host_sp.data();
        int ne = 0;
        for (size_t i = 0; i < n; ++i) ne += species[i] == 1;
        c->n_e = ne;
    }
    {
        std::vector<int> ne_cl(c->n_clouds, 0);
        for (int cl = 0; cl < c->n_clouds; ++cl)
            for (int i = c->cloud_start_h[cl]; i < c->cloud_start_h[cl + 1]; ++i)
                ne_cl[cl] += species[i] == 1;
        int rc = build_chunks(c, ne_cl);
        if (rc) return rc;
    }
    launch_deinterleave(dpos, c->n, c->st[k][0], c->st[k][1], c->st[k][2], c->s);
    launch_deinterleave(dvel, c->n, c->st[k][3], c->st[k][4], c->st[k][5], c->s);
    launch_iota(c->id[k], c->n, c->s);
    CK(cudaMemcpyAsync(c->sp_caller, c->sp[k], n, cudaMemcpyDeviceToDevice, c->s));
    CK(cudaMemsetAsync(c->sort.err, 0, sizeof(int), c->s));
    c->have_state = true;
    c->tree_valid = false;
    c->acc_valid = false;
    c->phi_valid = false;
    c->steps = 0;
    int rc = check_launch(c, "set_state");
    if (rc) return rc;
    if (!on_device) CK(cudaStreamSynchronize(c->s));
    return UCP_OK;
}

int ucp_get_state(ucp_ctx* c, double* pos, double* vel, int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    size_t n = (size_t)c->n;
    int k = c->cur;
    double* outs[2] = {pos, vel};
    for (int w = 0; w < 2; ++w) {
        if (!outs[w]) continue;
        double* dst = on_device ? outs[w] : c->stage + 3 * n * w;
        launch_scatter3(c->st[k][3 * w], c->st[k][3 * w + 1], c->st[k][3 * w + 2], c->id[k],
                        c->n, dst, c->s);
        if (!on_device)
            CK(cudaMemcpyAsync(outs[w], dst, 3 * n * sizeof(double), cudaMemcpyDeviceToHost,
                               c->s));
    }
    int rc = check_launch(c, "get_state");
    if (rc) return rc;
    if (!on_device) {
        CK(cudaStreamSynchronize(c->s));
        if ((rc = device_error(c))) return rc;
    }
    return UCP_OK;
}

int ucp_tree_build(ucp_ctx* c)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    if (c->tree_valid) return UCP_OK;
    return build(c);
}

int ucp_tree_force(ucp_ctx* c, double theta, double eps, double* acc, double* phi, int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    if (!c->tree_valid && (rc = build(c))) return rc;
    if ((rc = force(c, theta, eps, 0, phi != nullptr))) return rc;
    size_t n = (size_t)c->n;
    int k = c->cur;
    if (acc) {
        double* dst = on_device ? acc : c->stage;
        launch_scatter3(c->ax, c->ay, c->az, c->id[k], c->n, dst, c->s);
        if (!on_device)
            CK(cudaMemcpyAsync(acc, dst, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    }
    if (phi) {
        double* dst = on_device ? phi : c->stage + 3 * n;
        launch_scatter1(c->phi, c->id[k], c->n, dst, c->s);
        if (!on_device)
            CK(cudaMemcpyAsync(phi, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    }
    if ((rc = check_launch(c, "tree_force"))) return rc;
    if (!on_device) {
        CK(cudaStreamSynchronize(c->s));
        if ((rc = device_error(c))) return rc;
    }
    return UCP_OK;
}

// The split-step push; with store != NULL the positions after every electron
// substep are written there in caller order (n x 3 doubles per substep).
static int run_blocks(ucp_ctx* c, double dt_e, int kk, int64_t nblocks, double theta, double eps,
                      double* store)
{
    int rc;
    if (!c->acc_valid) {
        if (!c->tree_valid && (rc = build(c))) return rc;
        if ((rc = force(c, theta, eps, 0, false))) return rc;
    }
    const double dt_i = (double)kk * dt_e;
    const double h_i = 0.5 * dt_i, h_e = 0.5 * dt_e;
    int pend_i = 0, pend_e = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        int k = c->cur;
        launch_kick(c->st[k][3], c->st[k][4], c->st[k][5], c->ax, c->ay, c->az, c->sp[k], UCP_ION,
                    h_i, c->n, 1 + pend_i, c->s);
        pend_i = 0;
        for (int sub = 1; sub <= kk; ++sub) {
            k = c->cur;
            launch_kick(c->st[k][3], c->st[k][4], c->st[k][5], c->ax, c->ay, c->az, c->sp[k],
                        UCP_ELECTRON, h_e, c->n, 1 + pend_e, c->s);
            pend_e = 0;
            launch_drift(c->st[k][0], c->st[k][1], c->st[k][2], c->st[k][3], c->st[k][4],
                         c->st[k][5], dt_e, c->n, c->s);
            if ((rc = build(c))) return rc;
            // the walk over every particle also leaves phi for a following ucp_energy
            if ((rc = force(c, theta, eps, sub < kk, sub == kk))) return rc;
            pend_e = 1;
            if (store) {
                k = c->cur;
                launch_scatter3(c->st[k][0], c->st[k][1], c->st[k][2], c->id[k], c->n,
                                store + (size_t)3 * c->n * (size_t)(b * kk + sub - 1), c->s);
            }
        }
        pend_i = 1;
        c->steps += kk;
    }
    int k = c->cur;
    if (pend_e)
        launch_kick(c->st[k][3], c->st[k][4], c->st[k][5], c->ax, c->ay, c->az, c->sp[k],
                    UCP_ELECTRON, h_e, c->n, 1, c->s);
    if (pend_i)
        launch_kick(c->st[k][3], c->st[k][4], c->st[k][5], c->ax, c->ay, c->az, c->sp[k], UCP_ION,
                    h_i, c->n, 1, c->s);
    return check_launch(c, "step");
}

// One block of the push as a CUDA graph: captured on first use for (k, dt_e,
// theta, eps, buffer parity) on a private stream, replayed on the context's
// stream afterwards.  The block body is run_blocks with one block (no kick
// fusion across blocks, which changes no result).
static int run_block_graph(ucp_ctx* c, double dt_e, int kk, double theta, double eps)
{
    ucp_ctx::GraphEntry* hit = nullptr;
    for (auto& g : c->graphs)
        if (g.kk == kk && g.cur_in == c->cur && g.n_e == c->n_e &&
            g.n_chunks_all == c->n_chunks_all && g.n_chunks_e == c->n_chunks_e &&
            g.dt_e == dt_e && g.theta == theta && g.eps == eps && g.prof == c->prof)
            hit = &g;
    if (!hit) {
        if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking))
            return fail(c, UCP_ECUDA, "capture stream");
        const int cur0 = c->cur;
        const int64_t steps0 = c->steps, wt0 = c->walk_targets, wl0 = c->walk_launches;
        cudaStream_t orig = c->s;
        c->s = c->cap_stream;
        const unsigned long long l0 = g_launches.load();
        cudaGraph_t graph = nullptr;
        int rc = UCP_OK;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal)) {
            c->s = orig;
            return fail(c, UCP_ECUDA, "begin capture");
        }
        c->cap_prof = c->prof;
        c->cap_ev_used = 0;
        rc = run_blocks(c, dt_e, kk, 1, theta, eps, nullptr);
        c->cap_prof = false;
        cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
        c->s = orig;
        const unsigned long long nl = g_launches.load() - l0;
        g_launches.fetch_sub(nl);
        const int cur1 = c->cur;
        c->cur = cur0;
        c->steps = steps0;
        c->walk_targets = wt0;
        c->walk_launches = wl0;
        if (rc || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : fail(c, UCP_ECUDA, "capture of a step block failed");
        }
        // the event-record nodes, in the order their placeholder events were recorded
        std::vector<cudaGraphNode_t> ev_nodes(c->prof ? c->cap_ev_used : 0, nullptr);
        if (c->prof) {
            size_t nn = 0;
            cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(graph, nodes.data(), &nn);
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord)
                    continue;
                cudaEvent_t e;
                if (cudaGraphEventRecordNodeGetEvent(nd, &e) != cudaSuccess) continue;
                for (size_t i = 0; i < c->cap_ev_used; ++i)
                    if (c->cap_ev[i] == e) ev_nodes[i] = nd;
            }
            for (cudaGraphNode_t nd : ev_nodes)
                if (!nd || (ev_nodes.size() & 1)) {
                    cudaGraphDestroy(graph);
                    return fail(c, UCP_ECUDA, "profiled capture: event nodes not found");
                }
        }
        cudaGraphExec_t exec = nullptr;
        ec = cudaGraphInstantiate(&exec, graph, 0);
        if (ec != cudaSuccess) {
            cudaGraphDestroy(graph);
            return fail(c, UCP_ECUDA, "graph instantiation failed");
        }
        c->graphs.push_back({kk, cur0, cur1, c->n_e, c->n_chunks_all, c->n_chunks_e, dt_e, theta,
                             eps, c->prof, graph, exec, nl, ev_nodes});
        hit = &c->graphs.back();
    }
    if (hit->prof) {
        // point each walk's begin/end nodes at the next pair of the profiling pool
        for (size_t i = 0; i + 1 < hit->ev_nodes.size(); i += 2) {
            if (c->ev_used == c->ev.size()) {
                cudaEvent_t a, b;
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                c->ev.push_back({a, b});
            }
            CK(cudaGraphExecEventRecordNodeSetEvent(hit->exec, hit->ev_nodes[i],
                                                     c->ev[c->ev_used].first));
            CK(cudaGraphExecEventRecordNodeSetEvent(hit->exec, hit->ev_nodes[i + 1],
                                                     c->ev[c->ev_used].second));
            ++c->ev_used;
        }
    }
    CK(cudaGraphLaunch(hit->exec, c->s));
    count_launch((int)hit->launches);
    c->cur = hit->cur_out;
    c->steps += kk;
    c->tree_valid = true;
    c->acc_valid = true;
    c->phi_valid = true;
    c->phi_theta = theta;
    c->phi_eps = eps;
    c->walk_launches += kk;
    c->walk_targets += (int64_t)(kk - 1) * c->n_e + c->n;
    return UCP_OK;
}

// Times the FP32C walks of one block step (one over every particle, nine over
// the electrons) in each launch shape and keeps the fastest; results do not
// depend on the shape.
int ucp_autotune(ucp_ctx* c, double theta, double eps, int* best_shape, float* best_ms)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    if (c->precision != UCP_FP32C) {
        if (best_shape) *best_shape = 0;
        return UCP_OK;
    }
    if (!c->tree_valid && (rc = build(c))) return rc;
    const bool prof = c->prof;
    c->prof = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = 0;
    float best_t = 1e30f;
    int64_t wt = c->walk_targets, wl = c->walk_launches;
    unsigned long long st[2];
    CK(cudaMemcpyAsync(st, c->stats, sizeof(st), cudaMemcpyDeviceToHost, c->s));
    // cost of a shape: the walks of one block of 10 electron substeps (one over
    // every particle, nine over the electrons), best of three after a warm-up
    auto timed = [&](int electrons_only, float* ms) {
        CK(cudaEventRecord(e0, c->s));
        int r = force(c, theta, eps, electrons_only, false);
        CK(cudaEventRecord(e1, c->s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        return r;
    };
    for (int sh = 0; sh < walk_shape_count() && !rc; ++sh) {
        c->walk_shape = sh;
        float tbest = 1e30f;
        for (int rep = 0; rep < 4 && !rc; ++rep) {
            float t_all = 0.f, t_e = 0.f;
            rc = timed(0, &t_all);
            if (!rc && c->n_e > 0) rc = timed(1, &t_e);
            const float t = t_all + 9.f * t_e;
            if (rep > 0 && t < tbest) tbest = t;   // the first run warms caches
        }
        if (tbest < best_t) {
            best_t = tbest;
            best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpyAsync(c->stats, st, sizeof(st), cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    c->walk_targets = wt;
    c->walk_launches = wl;
    c->walk_shape = best;
    c->prof = prof;
    // the trial walks used this call's theta and eps: the next step recomputes
    // its first forces (identical to the cached ones when theta and eps agree)
    c->acc_valid = false;
    for (auto& g : c->graphs) {  // recapture with the new shape
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    c->graphs.clear();
    if (best_shape) *best_shape = best;
    if (best_ms) *best_ms = best_t;
    return rc;
}

int ucp_set_walk_shape(ucp_ctx* c, int shape)
{
    if (!c) return UCP_EINVAL;
    if (shape < 0 || shape >= walk_shape_count() || walk_shape_count() != UCP_WALK_SHAPES)
        return fail(c, UCP_EINVAL, "walk shape out of range");
    if (c->walk_shape != shape) {
        for (auto& g : c->graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
        }
        c->graphs.clear();
    }
    c->walk_shape = shape;
    return UCP_OK;
}

int ucp_set_graphs(ucp_ctx* c, int enable)
{
    if (!c) return UCP_EINVAL;
    c->use_graphs = enable != 0;
    return UCP_OK;
}

int ucp_step(ucp_ctx* c, double dt_e, int kk, int64_t n_electron_steps, double theta, double eps)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    if (!(dt_e > 0.0) || !std::isfinite(dt_e)) return fail(c, UCP_EINVAL, "dt_e must be > 0");
    if (kk < 1) return fail(c, UCP_EINVAL, "ion_substep_ratio must be >= 1");
    if (n_electron_steps < 0 || n_electron_steps % kk)
        return fail(c, UCP_EINVAL, "n_electron_steps must be a non-negative multiple of k");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    if (!c->use_graphs) return run_blocks(c, dt_e, kk, n_electron_steps / kk, theta, eps, nullptr);
    if (!c->acc_valid) {
        if (!c->tree_valid && (rc = build(c))) return rc;
        if ((rc = force(c, theta, eps, 0, false))) return rc;
    }
    for (int64_t b = 0; b < n_electron_steps / kk; ++b)
        if ((rc = run_block_graph(c, dt_e, kk, theta, eps))) return rc;
    return UCP_OK;
}

// Replace the positions and velocities (device, caller order) without the
// checks of ucp_set_state; species stay as set.
static void load_state(ucp_ctx* c, const double* dpos, const double* dvel)
{
    int k = c->cur;
    launch_deinterleave(dpos, c->n, c->st[k][0], c->st[k][1], c->st[k][2], c->s);
    launch_deinterleave(dvel, c->n, c->st[k][3], c->st[k][4], c->st[k][5], c->s);
    cudaMemcpyAsync(c->sp[k], c->sp_caller, (size_t)c->n, cudaMemcpyDeviceToDevice, c->s);
    launch_iota(c->id[k], c->n, c->s);
    c->tree_valid = false;
    c->acc_valid = false;
    c->phi_valid = false;
}

int ucp_grad_ke_electrons(ucp_ctx* c, double dt_e, int kk, int64_t n_steps, double theta,
                          double eps, int64_t checkpoint_every, double* loss, double* grad_x,
                          double* grad_v, int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    if (!(dt_e > 0.0) || !std::isfinite(dt_e) || kk < 1 || n_steps < kk || n_steps % kk ||
        checkpoint_every < kk || checkpoint_every % kk)
        return fail(c, UCP_EINVAL, "need k >= 1, n_steps and checkpoint_every multiples of k");
    if (c->potential != UCP_POT_PLUMMER) return fail(c, UCP_EINVAL, "adjoint: Plummer law only");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    const size_t n3 = (size_t)3 * c->n;
    const int64_t S = n_steps, C = checkpoint_every;
    const int64_t nseg = (S + C - 1) / C;
    // working memory of this call: checkpoints, one segment of positions, lambdas
    double *ck = nullptr, *seg = nullptr, *lx = nullptr, *lv = nullptr, *lam = nullptr,
           *lsorted = nullptr, *mu = nullptr, *adj = nullptr, *dloss = nullptr, *zero = nullptr;
    auto freeall = [&]() {
        for (double* p : {ck, seg, lx, lv, lam, lsorted, mu, adj, dloss, zero})
            if (p) cudaFree(p);
    };
    size_t adj_words = (size_t)c->t.cap * 12;
    if (cudaMalloc(&ck, sizeof(double) * n3 * 2 * (nseg + 1)) ||
        cudaMalloc(&seg, sizeof(double) * n3 * (C + 1)) || cudaMalloc(&lx, sizeof(double) * n3) ||
        cudaMalloc(&lv, sizeof(double) * n3) || cudaMalloc(&lam, sizeof(double) * n3) ||
        cudaMalloc(&lsorted, sizeof(double) * n3) || cudaMalloc(&mu, sizeof(double) * n3) ||
        cudaMalloc(&adj, sizeof(double) * adj_words) || cudaMalloc(&dloss, sizeof(double)) ||
        cudaMalloc(&zero, sizeof(double) * n3)) {
        cudaGetLastError();
        freeall();
        return fail(c, UCP_ENOMEM, "adjoint working memory");
    }
    auto snapshot = [&](double* dst) {
        int k = c->cur;
        launch_scatter3(c->st[k][0], c->st[k][1], c->st[k][2], c->id[k], c->n, dst, c->s);
        launch_scatter3(c->st[k][3], c->st[k][4], c->st[k][5], c->id[k], c->n, dst + n3, c->s);
    };
    const double h_e = 0.5 * dt_e, h_i = 0.5 * (double)kk * dt_e;
    int64_t steps0 = c->steps;
    // forward, checkpoints at g = 0, C, 2C, ...; the last segment's positions are
    // kept as the reverse sweep's first segment (no recomputation of it)
    snapshot(ck);
    for (int64_t sgi = 0; sgi < nseg; ++sgi) {
        int64_t len = std::min(C, S - sgi * C);
        const bool last = sgi == nseg - 1;
        if (last)
            cudaMemcpyAsync(seg, ck + 2 * n3 * sgi, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                            c->s);
        if ((rc = run_blocks(c, dt_e, kk, len / kk, theta, eps, last ? seg + n3 : nullptr))) break;
        snapshot(ck + 2 * n3 * (sgi + 1));
    }
    if (rc) {
        freeall();
        return rc;
    }
    launch_ke_seed(ck + 2 * n3 * nseg + n3, c->sp_caller, c->n, c->m[UCP_ELECTRON], lv, dloss,
                   c->s);
    cudaMemsetAsync(lx, 0, sizeof(double) * n3, c->s);
    cudaMemsetAsync(zero, 0, sizeof(double) * n3, c->s);
    WalkArgs a;
    // reverse: for g = S .. 1: adjoint of the kicks at X_g, then of drift g; X_0 last
    for (int64_t sgi = nseg - 1; sgi >= 0 && !rc; --sgi) {
        const int64_t g0 = sgi * C, len = std::min(C, S - g0);
        // seg[0] = X_{g0}; seg[j] = X_{g0 + j} (the last segment's from the forward run)
        if (sgi < nseg - 1) {
            load_state(c, ck + 2 * n3 * sgi, ck + 2 * n3 * sgi + n3);
            cudaMemcpyAsync(seg, ck + 2 * n3 * sgi, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                            c->s);
            if ((rc = run_blocks(c, dt_e, kk, len / kk, theta, eps, seg + n3))) break;
        }
        for (int64_t j = len; j >= (sgi == 0 ? 0 : 1); --j) {
            const int64_t g = g0 + j;
            // merged kicks that use a(X_g): electrons 2 h_e (1 at the ends), ions 2 h_i at
            // block boundaries (1 at the ends), none inside a block
            const bool endp = g == 0 || g == S;
            const double ce = (endp ? 1.0 : 2.0) * h_e;
            const double ci = (g % kk == 0) ? (endp ? 1.0 : 2.0) * h_i : 0.0;
            load_state(c, seg + n3 * (size_t)j, zero);
            if ((rc = build(c))) break;
            const int f32 = c->precision == UCP_FP32C;
            launch_mac_prepare(c->t, c->cube, theta, f32, c->s);
            int k = c->cur;
            launch_kick_lambda(lv, c->sp_caller, c->n, ce, ci, lam, c->s);
            launch_gather3(lam, c->id[k], c->n, lsorted, c->s);
            a.x = c->st[k][0];
            a.y = c->st[k][1];
            a.z = c->st[k][2];
            a.sp = c->sp[k];
            a.qsp = c->qsp;
            a.msp = c->msp;
            a.src32 = f32 ? c->src32 : nullptr;  // FP32C: the FP32 adjoint walk
            a.t = c->t;
            if (ci == 0.0 && c->n_e > 0) {
                // inside a block the ions' weights are zero: only the electrons'
                // accelerations carry adjoint weight, so only they are walked
                launch_select(c->sp[k], UCP_ELECTRON, c->n, c->tlist, c->scan_part,
                              c->tcount, c->s);
                a.targets = c->tlist;
                a.ntargets = c->n_e;
                a.chunks = c->chunks_e;
                a.nchunks = c->n_chunks_e;
            } else {
                a.targets = nullptr;
                a.ntargets = c->n;
                a.chunks = c->chunks_all;
                a.nchunks = c->n_chunks_all;
            }
            a.pos_off = c->pos_off;
            a.cubes = c->cube;
            a.eps2 = eps * eps;
            a.kelbg = 0;
            a.lambda = 1.0;
            a.work = c->work;
            a.err = c->sort.err;
            launch_walk_adjoint(a, lsorted, mu, adj, c->n, c->nsm, c->s);
            launch_scatter_add3(mu, c->id[k], c->n, lx, c->s);
            if (g > 0) launch_axpy3(lv, lx, dt_e, c->n, c->s);  // drift g
            if ((rc = check_launch(c, "adjoint"))) break;
        }
    }
    if (!rc) {
        double L = 0.0;
        cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (grad_x && cudaMemcpyAsync(grad_x, lx, sizeof(double) * n3, kind, c->s)) rc = UCP_ECUDA;
        if (grad_v && cudaMemcpyAsync(grad_v, lv, sizeof(double) * n3, kind, c->s)) rc = UCP_ECUDA;
        if (cudaMemcpyAsync(&L, dloss, sizeof(double), cudaMemcpyDeviceToHost, c->s)) rc = UCP_ECUDA;
        // leave the context at the end of the run
        load_state(c, ck + 2 * n3 * nseg, ck + 2 * n3 * nseg + n3);
        if (cudaStreamSynchronize(c->s)) rc = UCP_ECUDA;
        if (loss) *loss = L;
        c->steps = steps0 + S;
        if (rc) fail(c, rc, "adjoint copies failed");
    }
    cudaStreamSynchronize(c->s);
    freeall();
    if (!rc) rc = device_error(c);
    return rc;
}

// (d a / d x)^T lam at the current positions, the tree held fixed: the adjoint
// walk of the gradient call, on its own.
int ucp_accel_vjp(ucp_ctx* c, double theta, double eps, const double* lam_in, double* mu_out,
                  int on_device)
{
    if (!c || !lam_in || !mu_out) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    if (c->potential != UCP_POT_PLUMMER) return fail(c, UCP_EINVAL, "adjoint: Plummer law only");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    const size_t n3 = (size_t)3 * c->n;
    double *lam = nullptr, *lsorted = nullptr, *mu = nullptr, *adj = nullptr, *out = nullptr;
    auto freeall = [&]() {
        for (double* p : {lam, lsorted, mu, adj, out})
            if (p) cudaFree(p);
    };
    if (cudaMalloc(&lam, sizeof(double) * n3) || cudaMalloc(&lsorted, sizeof(double) * n3) ||
        cudaMalloc(&mu, sizeof(double) * n3) || cudaMalloc(&out, sizeof(double) * n3) ||
        cudaMalloc(&adj, sizeof(double) * (size_t)c->t.cap * 12)) {
        cudaGetLastError();
        freeall();
        return fail(c, UCP_ENOMEM, "adjoint working memory");
    }
    cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(lam, lam_in, sizeof(double) * n3, kin, c->s) ||
        cudaMemsetAsync(out, 0, sizeof(double) * n3, c->s)) {
        freeall();
        return fail(c, UCP_ECUDA, "adjoint input copy");
    }
    if (!c->tree_valid && (rc = build(c))) {
        freeall();
        return rc;
    }
    const int f32 = c->precision == UCP_FP32C;
    launch_mac_prepare(c->t, c->cube, theta, f32, c->s);
    const int k = c->cur;
    launch_gather3(lam, c->id[k], c->n, lsorted, c->s);
    WalkArgs a;
    a.x = c->st[k][0];
    a.y = c->st[k][1];
    a.z = c->st[k][2];
    a.sp = c->sp[k];
    a.qsp = c->qsp;
    a.msp = c->msp;
    a.src32 = f32 ? c->src32 : nullptr;
    a.t = c->t;
    a.targets = nullptr;
    a.ntargets = c->n;
    a.chunks = c->chunks_all;
    a.nchunks = c->n_chunks_all;
    a.pos_off = c->pos_off;
    a.cubes = c->cube;
    a.eps2 = eps * eps;
    a.kelbg = 0;
    a.lambda = 1.0;
    a.work = c->work;
    a.err = c->sort.err;
    launch_walk_adjoint(a, lsorted, mu, adj, c->n, c->nsm, c->s);
    launch_scatter_add3(mu, c->id[k], c->n, out, c->s);
    rc = check_launch(c, "adjoint walk");
    cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!rc && cudaMemcpyAsync(mu_out, out, sizeof(double) * n3, kout, c->s))
        rc = fail(c, UCP_ECUDA, "adjoint output copy");
    cudaStreamSynchronize(c->s);
    freeall();
    if (!rc) rc = device_error(c);
    return rc;
}

int ucp_energy(ucp_ctx* c, double theta, double eps, double out[6])
{
    if (!c || !out) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    int rc = valid_walk_args(c, theta, eps);
    if (rc) return rc;
    if (!c->tree_valid && (rc = build(c))) return rc;
    if (!(c->phi_valid && c->phi_theta == theta && c->phi_eps == eps) &&
        (rc = force(c, theta, eps, 0, true)))
        return rc;
    int k = c->cur;
    double r[6] = {0, 0, 0, 0, 0, 0};
    if (c->n_clouds == 1) {
        launch_energy(c->st[k][3], c->st[k][4], c->st[k][5], c->phi, c->sp[k], c->qsp, c->msp,
                      c->n, c->en_part, c->en_nblk, c->en_out, c->s);
        CK(cudaMemcpyAsync(r, c->en_out, sizeof(r), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
    } else {
        launch_energy_clouds(c->st[k][3], c->st[k][4], c->st[k][5], c->phi, c->sp[k], c->qsp,
                             c->msp, c->cloud_start, c->n_clouds, c->en_out, c->s);
        std::vector<double> per(6 * (size_t)c->n_clouds);
        CK(cudaMemcpyAsync(per.data(), c->en_out, sizeof(double) * per.size(),
                           cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        c->cloud_energy = per;
        for (int cl = 0; cl < c->n_clouds; ++cl)
            for (int j = 0; j < 6; ++j) r[j] += per[6 * cl + j];
    }
    if ((rc = check_launch(c, "energy"))) return rc;
    if ((rc = device_error(c))) return rc;
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
    out[3] = r[0] + r[1] + r[2];
    out[4] = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
    out[5] = (double)c->steps;
    return UCP_OK;
}

int ucp_energy_clouds(ucp_ctx* c, double theta, double eps, double* out)
{
    if (!c || !out) return UCP_EINVAL;
    double tot[6];
    int rc = ucp_energy(c, theta, eps, tot);
    if (rc) return rc;
    for (int cl = 0; cl < c->n_clouds; ++cl) {
        const double* r = c->n_clouds == 1 ? nullptr : &c->cloud_energy[6 * cl];
        double v[6];
        if (r) {
            for (int j = 0; j < 6; ++j) v[j] = r[j];
        }
        double* o = out + 6 * (size_t)cl;
        if (!r) {
            for (int j = 0; j < 6; ++j) o[j] = tot[j];
            continue;
        }
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
        o[3] = v[0] + v[1] + v[2];
        o[4] = std::sqrt(v[3] * v[3] + v[4] * v[4] + v[5] * v[5]);
        o[5] = (double)c->steps;
    }
    return UCP_OK;
}

int ucp_get_cubes(ucp_ctx* c, double* out)
{
    if (!c || !out) return UCP_EINVAL;
    if (!c->tree_valid) return fail(c, UCP_ESTATE, "no tree built");
    std::vector<Cube> cb(c->n_clouds);
    CK(cudaMemcpyAsync(cb.data(), c->cube, sizeof(Cube) * cb.size(), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    for (int cl = 0; cl < c->n_clouds; ++cl) {
        out[4 * cl] = cb[cl].c[0];
        out[4 * cl + 1] = cb[cl].c[1];
        out[4 * cl + 2] = cb[cl].c[2];
        out[4 * cl + 3] = cb[cl].L;
    }
    return UCP_OK;
}

int ucp_stats(ucp_ctx* c, int64_t out[8], int reset)
{
    if (!c || !out) return UCP_EINVAL;
    unsigned long long s2[2] = {0, 0};
    int nn = 0, md = 0;
    CK(cudaMemcpyAsync(s2, c->stats, sizeof(s2), cudaMemcpyDeviceToHost, c->s));
    if (c->tree_valid) {
        CK(cudaMemcpyAsync(&nn, c->t.nnodes, sizeof(int), cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(&md, c->t.maxdepth, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    }
    CK(cudaStreamSynchronize(c->s));
    int derr = device_error(c);
    out[0] = (int64_t)s2[0];
    out[1] = (int64_t)s2[1];
    out[2] = c->walk_targets;
    out[3] = c->walk_launches;
    out[4] = nn;
    out[5] = md;
    unsigned long long gl = g_launches.load();
    out[6] = (int64_t)(gl - c->launch_base);
    out[7] = 0;
    if (reset) {
        c->launch_base = gl;
        CK(cudaMemsetAsync(c->stats, 0, sizeof(s2), c->s));
        CK(cudaStreamSynchronize(c->s));
        c->walk_targets = 0;
        c->walk_launches = 0;
    }
    return derr;
}

int ucp_get_cube(ucp_ctx* c, double out[4])
{
    if (!c || !out) return UCP_EINVAL;
    if (!c->tree_valid) return fail(c, UCP_ESTATE, "no tree built");
    Cube cb;
    CK(cudaMemcpyAsync(&cb, c->cube, sizeof(cb), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    out[0] = cb.c[0];
    out[1] = cb.c[1];
    out[2] = cb.c[2];
    out[3] = cb.L;
    return UCP_OK;
}

int ucp_get_sorted(ucp_ctx* c, uint64_t* keys, uint32_t* ids, int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!c->tree_valid) return fail(c, UCP_ESTATE, "no tree built");
    size_t n = (size_t)c->n;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (keys) CK(cudaMemcpyAsync(keys, c->key[c->sorted_buf], n * 8, kind, c->s));
    if (ids) CK(cudaMemcpyAsync(ids, c->id[c->cur], n * 4, kind, c->s));
    if (!on_device) CK(cudaStreamSynchronize(c->s));
    return UCP_OK;
}

static unsigned int host_compact3(unsigned long long x)
{
    unsigned int r = 0;
    for (int b = 0; b < 21; ++b) r |= (unsigned int)((x >> (3 * b)) & 1ull) << b;
    return r;
}

int ucp_get_tree(ucp_ctx* c, int64_t* nnodes, int64_t cap, int32_t* topo, int8_t* is_leaf,
                 double* geom)
{
    if (!c || !nnodes) return UCP_EINVAL;
    if (!c->tree_valid) return fail(c, UCP_ESTATE, "no tree built");
    int nn = 0;
    std::vector<Cube> cubes(c->n_clouds);
    CK(cudaMemcpyAsync(&nn, c->t.nnodes, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(cubes.data(), c->cube, sizeof(Cube) * cubes.size(), cudaMemcpyDeviceToHost,
                       c->s));
    CK(cudaStreamSynchronize(c->s));
    *nnodes = nn;
    if (!topo && !is_leaf && !geom) return UCP_OK;
    if (cap < nn) return fail(c, UCP_EINVAL, "capacity smaller than the box count");
    std::vector<int4> info(nn);
    std::vector<int> dl(nn);
    std::vector<unsigned long long> cell(nn);
    std::vector<double> mom((size_t)nn * kMom);
    CK(cudaMemcpyAsync(info.data(), c->t.info, sizeof(int4) * nn, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(dl.data(), c->t.depth_leaf, sizeof(int) * nn, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(cell.data(), c->t.cell, 8 * (size_t)nn, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(mom.data(), c->t.mom, sizeof(double) * kMom * nn, cudaMemcpyDeviceToHost,
                       c->s));
    CK(cudaStreamSynchronize(c->s));
    for (int i = 0; i < nn; ++i) {
        int d = dl[i] & 255;
        if (topo) {
            topo[4 * i] = info[i].x;
            topo[4 * i + 1] = info[i].y;
            topo[4 * i + 2] = info[i].z;
            topo[4 * i + 3] = d;
        }
        if (is_leaf) is_leaf[i] = (dl[i] & 256) ? 1 : 0;
        if (geom) {
            const int cl = (int)(std::upper_bound(c->cloud_start_h.begin(), c->cloud_start_h.end(),
                                                  info[i].x) - c->cloud_start_h.begin()) - 1;
            const Cube& cb = cubes[cl];
            double* g = geom + 20 * (size_t)i;
            double s = std::ldexp(cb.L, -d);
            unsigned int ic[3] = {host_compact3(cell[i]), host_compact3(cell[i] >> 1),
                                  host_compact3(cell[i] >> 2)};
            for (int a = 0; a < 3; ++a) {
                volatile double lo = cb.c[a] - cb.L * 0.5;
                volatile double off = ((double)ic[a] + 0.5) * s;
                g[a] = lo + off;
            }
            g[3] = s;
            const double* m = mom.data() + (size_t)i * kMom;
            g[4] = m[MS0];
            g[5] = m[MM];
            for (int a = 0; a < 3; ++a) g[6 + a] = m[MC + a];
            for (int a = 0; a < 3; ++a) g[9 + a] = m[MD + a];
            for (int a = 0; a < 6; ++a) g[12 + a] = m[MQ + a];
            g[18] = m[MDELTA];
            g[19] = 0.0;
        }
    }
    return UCP_OK;
}

int ucp_get_counts(ucp_ctx* c, int32_t* p2p, int32_t* m2p, int on_device)
{
    if (!c) return UCP_EINVAL;
    if (!c->have_state) return fail(c, UCP_ESTATE, "no state");
    size_t n = (size_t)c->n;
    int k = c->cur;
    int32_t* outs[2] = {p2p, m2p};
    const int* srcs[2] = {c->cnt_p2p, c->cnt_m2p};
    for (int w = 0; w < 2; ++w) {
        if (!outs[w]) continue;
        int* dst = on_device ? outs[w] : c->stage_int + n * w;
        launch_scatter_int(srcs[w], c->id[k], c->n, dst, c->s);
        if (!on_device)
            CK(cudaMemcpyAsync(outs[w], dst, n * 4, cudaMemcpyDeviceToHost, c->s));
    }
    int rc = check_launch(c, "get_counts");
    if (rc) return rc;
    if (!on_device) CK(cudaStreamSynchronize(c->s));
    return UCP_OK;
}

int ucp_selftest_wait_timeout(ucp_ctx* c)
{
    if (!c) return UCP_EINVAL;
    CK(cudaStreamSynchronize(c->s));
    CK(cudaMemsetAsync(c->sort.err, 0, sizeof(int), c->s));
    if (sort_selftest_timeout(c->sort, c->s)) return fail(c, UCP_ECUDA, "self-test launch failed");
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->sort.err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    CK(cudaMemsetAsync(c->sort.err, 0, sizeof(int), c->s));
    CK(cudaStreamSynchronize(c->s));
    return e ? UCP_ETIMEOUT : UCP_OK;
}

int ucp_profile(ucp_ctx* c, int enable)
{
    if (!c) return UCP_EINVAL;
    c->prof = enable != 0;
    return UCP_OK;
}

int ucp_profile_read(ucp_ctx* c, double* walk_ms, int64_t* launches)
{
    if (!c) return UCP_EINVAL;
    CK(cudaStreamSynchronize(c->s));
    double tot = 0.0;
    for (size_t i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[i].first, c->ev[i].second));
        tot += ms;
    }
    if (walk_ms) *walk_ms = tot;
    if (launches) *launches = (int64_t)c->ev_used;
    c->ev_used = 0;
    return UCP_OK;
}

}  // extern "C"
