/*
 * ucp.h -- C ABI of the GB300 two-component plasma TREE library (libucp.so).
 *
 * The library evaluates the Coulomb force on the electrons and ions of an
 * open-boundary two-component plasma with the TREE method of Jeon, Kress,
 * Collins and Gronbech-Jensen (arXiv 0709.3331), Sec. 3, and advances the
 * particles with the velocity Verlet push of Sec. 2, electrons on a short
 * substep and ions on k of them.  One context = one particle set on one GPU.
 *
 * Conventions for every call:
 *   - Return 0 (UCP_OK) on success or a negative UCP_E* code; no call throws
 *     or aborts.  ucp_strerror() names the code; ucp_last_error() returns a
 *     message about the most recent failure in this context.
 *   - Arrays are in the caller's particle order (index i = the i-th particle
 *     handed to ucp_set_state); the library keeps its own copy in key order.
 *   - pos / vel / acc are N x 3 row-major double (x, y, z of particle 0 first).
 *   - on_device = 1: the pointer is CUDA device memory (e.g. a torch CUDA
 *     tensor's data_ptr) read or written in stream order on the context's
 *     stream and the call returns after enqueueing.  on_device = 0: host
 *     memory; the call copies and synchronises the stream before returning.
 *   - Units are reduced: Coulomb constant 1 (Eq. 2 with e^2/(4 pi eps0) = 1),
 *     so the pair potential is q_i q_j / sqrt(r^2 + eps^2) (Eq. 1 with
 *     Plummer softening eps).
 *   - A context is not thread-safe; different contexts are independent.
 *   - The caller owns every pointer it passes; the library owns the context
 *     and the device memory it allocates in ucp_create (freed by ucp_destroy).
 */
#ifndef UCP_H
#define UCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    UCP_OK = 0,
    UCP_EINVAL = -1,      /* bad argument (null pointer, size, theta, eps, dt, k) */
    UCP_ENOMEM = -2,      /* device or host allocation failed */
    UCP_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
    UCP_ENONFINITE = -4,  /* a position or velocity is NaN or infinite */
    UCP_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
    UCP_ESTATE = -6       /* call order: no state set yet */
};

enum { UCP_FP64 = 0, UCP_FP32C = 1 };  /* arithmetic of the force walk */
/* Direct-pair law: UCP_POT_PLUMMER = q_i q_j / sqrt(r^2 + eps^2) for every pair;
 * UCP_POT_KELBG = the Kelbg form q_i q_j (1 - exp(-r/lambda_ei)) / r of Sec. 2.1
 * Eq. 3 for electron-ion pairs (lambda_ei fixed, as Sec. 2.1 does), softened
 * Coulomb for like pairs; multipoles of accepted boxes stay Coulomb in both
 * (the exponential term is negligible in the far field, Sec. 2.1). */
enum { UCP_POT_PLUMMER = 0, UCP_POT_KELBG = 1 };
enum { UCP_ION = 0, UCP_ELECTRON = 1 }; /* species codes */

typedef struct ucp_ctx ucp_ctx;

typedef struct {
    int64_t n;          /* particles, 1 <= n <= 2^31 - 1 */
    int32_t leaf_cap;   /* a box with at most leaf_cap particles is a leaf
                           (Sec. 3 subdivides "until every box contains no more
                           than one particle": leaf_cap = 1); 1..1024 */
    int32_t precision;  /* UCP_FP64 or UCP_FP32C (FP32 node-relative arithmetic,
                           compensated sums, FP64 state and results) */
    double q[2];        /* charge per species [ion, electron] */
    double m[2];        /* mass per species, > 0 */
    void* cuda_stream;  /* cudaStream_t the context works on (NULL = legacy) */
    int32_t potential;  /* UCP_POT_PLUMMER (0) or UCP_POT_KELBG (needs q[0] != q[1]) */
    int32_t reserved;   /* 0 */
    double lambda_ei;   /* Kelbg length, > 0 (reduced units); ignored for Plummer */
} ucp_params;

/* Create a context for params->n particles and allocate all device memory
 * it will need (nothing is allocated later).  *out is set on success. */
int ucp_create(ucp_ctx** out, const ucp_params* params);

/* Ensemble of n_clouds independent clouds (1 <= n_clouds <= UCP_MAX_CLOUDS) in
 * one context: cloud c holds sizes[c] >= 1 particles, at caller indices
 * [sizes[0] + ... + sizes[c-1], ... + sizes[c]).  Clouds do not interact; each
 * has its own enclosing cube and TREE (Sec. 3), and every call below works on
 * all clouds at once, one kernel launch per stage for the whole ensemble (the
 * walk is one persistent launch over all clouds' targets).  params->n must be 0
 * or the total; the other parameters are common to all clouds. */
#define UCP_MAX_CLOUDS 256
int ucp_create_batch(ucp_ctx** out, const ucp_params* params, int32_t n_clouds,
                     const int64_t* sizes);

/* Free the context and its device memory (NULL is allowed). */
void ucp_destroy(ucp_ctx* ctx);

/* Copy in positions, velocities (N x 3) and species (N, values 0 or 1).
 * Rejects non-finite values with UCP_ENONFINITE and species outside {0,1}
 * with UCP_EINVAL.  Invalidates the tree and the stored accelerations and
 * resets the step counter. */
int ucp_set_state(ucp_ctx* ctx, const double* pos, const double* vel,
                  const int8_t* species, int on_device);

/* Copy out positions and velocities in the caller's order (either may be NULL). */
int ucp_get_state(ucp_ctx* ctx, double* pos, double* vel, int on_device);

/* Sec. 3 TREE construction on the current positions: enclosing cube, Morton
 * keys (21 bits per axis), stable key sort (ties by particle index), octree
 * boxes as key prefixes in pre-order, and moments of every box (monopole,
 * |q|-weighted centroid, dipole, second moment). */
int ucp_tree_build(ucp_ctx* ctx);

/* Sec. 3 particle-TREE interaction on every particle with the opening
 * criterion of Eq. 5 (s/theta + delta < d; 0 <= theta <= 1) and softening
 * eps >= 0.  Builds the tree first if the positions changed since the last
 * build.  acc (N x 3, = q_t E_t / m_t) and phi (N, potential at the
 * particle, no self term) may each be NULL.  Also stores the accelerations
 * for a following ucp_step. */
int ucp_tree_force(ucp_ctx* ctx, double theta, double eps, double* acc, double* phi,
                   int on_device);

/* Sec. 2 velocity Verlet with electron substeps: n_electron_steps / k blocks
 * (n_electron_steps must be a multiple of k = ion_substep_ratio >= 1).  One
 * block, dt_i = k dt_e:
 *   ions v += dt_i/2 a;  k times { electrons v += dt_e/2 a; all x += dt_e v;
 *   rebuild the tree; a of the electrons (of every particle on the k-th);
 *   electrons v += dt_e/2 a };  ions v += dt_i/2 a.
 * k = 1 is plain velocity Verlet.  Accelerations of the current positions
 * are computed first when none are stored. */
int ucp_step(ucp_ctx* ctx, double dt_e, int ion_substep_ratio, int64_t n_electron_steps,
             double theta, double eps);

/* Gradient of the electron kinetic energy after a run.  From the current state
 * (x0, v0), advances n_steps electron substeps exactly as ucp_step(dt_e, k,
 * n_steps, theta, eps) and returns *loss = L = sum over electrons of m v^2 / 2 at
 * the end, grad_x = dL/dx0 and grad_v = dL/dv0 (N x 3, caller order; either may
 * be NULL).  Reverse mode: the discrete adjoint of every kick and drift, and at
 * every substep the adjoint of the TREE force with the tree held fixed (the same
 * boxes as the forward walk), evaluated in FP64 (FP64 contexts) or in the FP32
 * node-relative form with FP64 accumulation of the scatter (FP32C contexts); the state is kept every
 * checkpoint_every substeps (a multiple of k) and each stretch is recomputed
 * forward before it is reversed.  The context ends in the state after the run.
 * This call allocates its working memory (about (n_steps / checkpoint_every +
 * checkpoint_every) x 48 N bytes plus 96 bytes per box) and frees it before it
 * returns.  Plummer law only (UCP_EINVAL for Kelbg contexts).  Source-side
 * sums use atomic adds: gradients may differ between runs in the last bits. */
/* The Hessian-vector walk on its own: mu = (d a / d x)^T lam for the TREE
 * accelerations a (N x 3, = q E / m, Sec. 3 with the Eq. 5 criterion) at the
 * current positions, the tree held fixed (the boxes a forward walk with theta
 * accepts or opens), for a caller-order vector lam (N x 3); mu is N x 3 in caller
 * order.  Pair and multipole terms are differentiated on both sides (targets,
 * and sources through the box moments and centres), in FP64 (FP64 contexts) or
 * the FP32 node-relative form (FP32C).  Allocates its working memory (72 bytes
 * per particle plus 96 per box) and frees it before returning; synchronises the
 * stream.  Plummer law only (UCP_EINVAL for Kelbg contexts); atomic source
 * sums: results may differ between runs in the last bits. */
int ucp_accel_vjp(ucp_ctx* ctx, double theta, double eps, const double* lam, double* mu,
                  int on_device);

int ucp_grad_ke_electrons(ucp_ctx* ctx, double dt_e, int ion_substep_ratio, int64_t n_steps,
                          double theta, double eps, int64_t checkpoint_every, double* loss,
                          double* grad_x, double* grad_v, int on_device);

/* enable != 0: ucp_step runs every block of k electron substeps as one CUDA graph,
 * captured on a private stream the first time a block with these (k, dt_e, theta,
 * eps) starts from a given state buffer, and replayed on the context's stream
 * afterwards (the results are identical to the stream-ordered launches; kernel
 * timing with ucp_profile turns it off).  Useful where launch overhead matters
 * (small clouds, ensembles). */
int ucp_set_graphs(ucp_ctx* ctx, int enable);

/* Autotuner of the FP32C walk: times, in each launch shape the library has
 * (threads per block x resident blocks per SM, sources through L1 or staged in
 * shared memory), the walks of one block of 10 electron substeps on the current
 * state (one walk over every particle and nine over the electrons; best of three
 * after a warm-up) and keeps the fastest shape for this context (returned in
 * *best_shape, that block's walk time in ms in *best_ms; either may be NULL).
 * Results do not depend on the shape.  FP64 contexts keep their single shape. */
int ucp_autotune(ucp_ctx* ctx, double theta, double eps, int* best_shape, float* best_ms);

/* Number of FP32C walk launch shapes, and a call that sets one directly
 * (0 = the default of 128 threads x 7 blocks per SM, leaf sources read
 * through L1; UCP_EINVAL outside
 * [0, UCP_WALK_SHAPES)).  The trial walks of ucp_autotune overwrite the forces and
 * interaction counts read by ucp_get_counts, and the next ucp_step recomputes its
 * first forces. */
#define UCP_WALK_SHAPES 10
int ucp_set_walk_shape(ucp_ctx* ctx, int shape);

/* Sec. 5 observables of the current state: out = {KE_ion, KE_electron, PE,
 * E = KE + PE, |P| (total momentum), electron steps taken}.  PE is
 * (1/2) sum_t q_t phi_t with the tree potential; the walk over all particles
 * that ends every ucp_step block already leaves phi, so after a step with the
 * same theta and eps this is a reduction only, otherwise one walk runs first. */
int ucp_energy(ucp_ctx* ctx, double theta, double eps, double out[6]);

/* Per-cloud observables of an ensemble: out[6 c + j] as ucp_energy's out[j]
 * for cloud c (n_clouds x 6 doubles); ucp_energy returns the sums (and |P| of
 * the total momentum). */
int ucp_energy_clouds(ucp_ctx* ctx, double theta, double eps, double* out);

/* Counters: out = {direct pairs, multipole evaluations, walk targets, walk
 * launches} summed since the last reset, {boxes, deepest depth} of the last
 * tree, {CUDA kernels launched by this library (all contexts of the process)
 * since the last reset, 0}.  reset != 0 zeroes the summed counters after
 * reading. */
int ucp_stats(ucp_ctx* ctx, int64_t out[8], int reset);

/* Inspection of the last build (tests): enclosing cube {centre xyz, side};
 * key-sorted 63-bit Morton keys and the caller index of each sorted slot;
 * box table in pre-order (host arrays of capacity cap >= *nnodes, else
 * UCP_EINVAL with *nnodes set): topo (cap x 4 int32 {begin, end, next,
 * depth}; begin/end index key-sorted slots, next = first box after the
 * subtree), is_leaf (cap int8), geom (cap x 20 double {centre xyz, side, S0,
 * M, c xyz, D xyz, Q xx xy xz yy yz zz, delta, 0}); any array may be NULL.
 * ucp_get_counts: direct pairs and multipole evaluations per particle in the
 * last walk, in the caller's order (0 for particles that were not targets). */
int ucp_get_cube(ucp_ctx* ctx, double out[4]);
int ucp_get_cubes(ucp_ctx* ctx, double* out); /* n_clouds x 4: every cloud's cube */
int ucp_get_sorted(ucp_ctx* ctx, uint64_t* keys, uint32_t* ids, int on_device);
int ucp_get_tree(ucp_ctx* ctx, int64_t* nnodes, int64_t cap, int32_t* topo,
                 int8_t* is_leaf, double* geom);
int ucp_get_counts(ucp_ctx* ctx, int32_t* p2p, int32_t* m2p, int on_device);

/* Failure-path self-test: runs one pass of the key sort as a lone block whose
 * predecessor never publishes, so its bounded wait runs out.  Returns
 * UCP_ETIMEOUT when the wait gave up and raised the error flag as it must (the
 * flag is cleared again and the context stays usable), UCP_OK if it did not. */
int ucp_selftest_wait_timeout(ucp_ctx* ctx);

/* Kernel timing: when enabled, the walk kernels are bracketed by CUDA events
 * on the context's stream; read returns {total ms, launches} of the walk since
 * the last read (synchronises the stream). */
int ucp_profile(ucp_ctx* ctx, int enable);
int ucp_profile_read(ucp_ctx* ctx, double* walk_ms, int64_t* walk_launches);

const char* ucp_strerror(int code);
const char* ucp_last_error(ucp_ctx* ctx);

/* Throughput of the arithmetic units the tree walk is bound by, measured on the
 * current device (no counterpart in the paper; it gives the walk's roofline a
 * denominator measured at the clocks of the run).  out = {FP32 FMA TFLOP/s,
 * packed FP32x2 FMA TFLOP/s, reciprocal square roots per second / 1e9, FP64
 * FMA TFLOP/s} (an FMA counts as 2 flops).  Runs about 0.1 s of kernels on
 * stream and synchronises it; allocates and frees a small scratch buffer.
 * UCP_EINVAL for out == NULL, UCP_ENOMEM, UCP_ECUDA. */
int ucp_measure_peaks(double out[4], void* stream);

/* Enclosing cube without any allocation.  The paper has no counterpart: this
 * is a service for callers that must not allocate GPU memory at this point --
 * for example code running while a CUDA graph is being captured (where
 * cudaMalloc is not allowed), code that works under a fixed device-memory
 * budget owned by another allocator, or real-time loops that forbid
 * allocation after start-up.  It computes the same cube as ucp_tree_build
 * (centre = (min + max) / 2 per axis, side = largest extent * (1 + 2^-20),
 * side 1 when all particles coincide) from pos (device, N x 3 double) into
 * cube_out (device, 4 doubles {centre x, y, z, side}), enqueued on stream
 * (cudaStream_t, NULL = legacy stream); it returns after enqueueing.
 * It calls no cudaMalloc or cudaFree: its per-tile partial results live in a
 * fixed array in the library's device memory (UCP_STATIC_MAX_N /
 * UCP_STATIC_TILE slots of 6 64-bit words, 48 KB, present on every GPU that
 * loads the library until the process exits).  N outside [1, UCP_STATIC_MAX_N]
 * returns UCP_EINVAL; a failed CUDA call returns UCP_ECUDA.  Min and max are
 * taken exactly as ucp_tree_build takes them, so the two cubes agree bit for
 * bit, signed zeros included; a NaN coordinate (which ucp_set_state refuses)
 * makes that axis's centre NaN here.
 * The first call on a device looks up that array's device address, with that
 * device current, and keeps it with the CUDA context it belongs to; a call in
 * another context (after a device reset, say) looks it up again.  Make the
 * first call on each device, and the first after a reset, before any stream
 * capture.  All calls share the one array and each call overwrites the slots
 * it uses, so calls that may run at the same time on the GPU (different
 * streams without ordering between them) race and must be serialised. */
#define UCP_STATIC_TILE 2048
#define UCP_STATIC_MAX_N (1024 * UCP_STATIC_TILE)
int ucp_root_cube_static(const double* pos, int64_t n, double* cube_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UCP_H */
