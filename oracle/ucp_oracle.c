/*
 * ucp_oracle.c -- plain, slow FP64 CPU oracle for the two-component plasma
 * TREE method (Jeon, Kress, Collins, Gronbech-Jensen, arXiv 0709.3331).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it is used by tests/, by the smoke check and by the
 * benchmark's CPU-baseline leg.  It shares no code, header or constant table
 * with the CUDA library; the two meet only through the seeded input arrays.
 *
 * What it computes (all in IEEE double, compiled with -ffp-contract=off so
 * that x86 and Arm give the same bits):
 *   - direct O(N^2) sum of the Plummer-softened Coulomb interaction
 *     (Sec. 2.1, Eq. 1-2, with e^2/(4 pi eps0) = 1 in reduced units);
 *   - the serial TREE of Sec. 3: enclosing cube, recursive eight-way
 *     subdivision until a box holds at most leaf_cap particles (the paper
 *     uses one), pseudo-particles, the opening criterion of Eq. 5, and the
 *     particle-tree interaction walked in pre-order;
 *   - the electron/ion split-step velocity Verlet push (Sec. 2) that calls
 *     the force every electron substep;
 *   - kinetic / potential energy and momentum (Sec. 5).
 *
 * Readings of the paper that this file fixes (the paper is silent or loose):
 *   R1  interaction: V = q_i q_j / sqrt(r^2 + eps^2) for every pair (Plummer
 *       softening replaces the Kelbg form of Eq. 3 for the e-i pair).
 *   R2  enclosing cube: centre = (min+max)/2 per axis, side L = (largest
 *       extent) * (1 + 2^-20); L = 1 when all particles coincide.
 *   R3  integer cell coordinates k = floor((x - lo) * (2^21 / L)) clamped to
 *       [0, 2^21 - 1] with lo = centre - L/2 and the scale 2^21 / L rounded
 *       once (even subdivision of the cube); a box at depth d holds the
 *       particles whose k agree in their top d bits; depth is capped at 21,
 *       so coincident particles end in one (fat) leaf.
 *   R4  pseudo-particle position (Sec. 3, "interpolated ... depending on the
 *       charge ratio") = |q|-weighted centroid c, since the signed charge of a
 *       neutral box is zero.  The expansion about c keeps monopole M, dipole
 *       D = sum q (x - c) and raw second moment Q = sum q (x-c)(x-c)^T.
 *   R5  opening criterion Eq. 5, s/theta + delta < d, with s the box side,
 *       delta = |c - box centre|, d = |x_t - c|; evaluated as
 *       (s/theta + delta)^2 < d^2 (same truth value, no square root);
 *       theta = 0 never accepts.  Leaves are tested too; a leaf that passes
 *       is applied as a multipole.
 *   R6  the multipole of a box on a target is the Taylor expansion of the
 *       softened kernel g(R) = (R^2 + eps^2)^(-1/2) about c through second
 *       order; the direct interaction skips j == t (no self term).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXDEPTH 21
#define ORC_KMAX ((uint32_t)1 << ORC_MAXDEPTH) /* 2^21 cells per axis */

/* ------------------------------------------------------------------ */
/* Interaction law of a direct pair.  g_kelbg = 0: Plummer-softened Coulomb for
 * every pair (R1).  g_kelbg = 1: the Kelbg form of Sec. 2.1 Eq. 3 for an
 * electron-ion pair, V = q_i q_j (1 - exp(-r/lambda)) / r with lambda fixed
 * (Sec. 2.1 fixes lambda_ei to one value instead of the thermal wavelength),
 * and bare (softened) Coulomb for like pairs; multipoles stay Coulomb, since the
 * exponential term is negligible in the far field (Sec. 2.1). */
static int g_kelbg = 0;
static double g_lambda = 1.0;

void orc_set_potential(int kelbg, double lambda)
{
    g_kelbg = kelbg;
    g_lambda = lambda;
}

/* Adds the field at xt due to a charge qj at xj (field = force per unit target
 * charge) and the potential.  unlike = the two particles are of different
 * species. */
static void pair_field(const double xt[3], const double xj[3], double qj, int unlike,
                       double eps2, double E[3], double* phi)
{
    double dx = xt[0] - xj[0];
    double dy = xt[1] - xj[1];
    double dz = xt[2] - xj[2];
    if (g_kelbg && unlike) {
        /* V/q_t = qj (1 - e)/r, e = exp(-r/lambda);
         * E = -grad = qj r_vec [(1 - e)/r^3 - e/(lambda r^2)] */
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r == 0.0) { /* limit r -> 0: potential qj/lambda, no force */
            *phi += qj / g_lambda;
            return;
        }
        double u = r / g_lambda;
        double e = exp(-u);
        double one_minus_e = -expm1(-u);
        double f = (one_minus_e / (r * r * r)) - e / (g_lambda * r * r);
        E[0] += qj * dx * f;
        E[1] += qj * dy * f;
        E[2] += qj * dz * f;
        *phi += qj * one_minus_e / r;
        return;
    }
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double rinv3 = rinv * rinv * rinv;
    E[0] += qj * dx * rinv3;
    E[1] += qj * dy * rinv3;
    E[2] += qj * dz * rinv3;
    *phi += qj * rinv;
}

/* Direct O(N^2) sum (Sec. 3: "all pair-wise calculations").  Targets are
 * tidx[0..nt) (or all particles when tidx is NULL, nt = n).  Outputs per
 * listed target: field E (n_t x 3) and potential phi. */
void orc_direct(int64_t n, const double* pos, const int8_t* species,
                const double q[2], double eps, const int64_t* tidx,
                int64_t nt, double* E_out, double* phi_out, int nthreads)
{
    double eps2 = eps * eps;
    if (!tidx) nt = n;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t a = 0; a < nt; ++a) {
        int64_t t = tidx ? tidx[a] : a;
        double E[3] = {0.0, 0.0, 0.0}, phi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == t) continue;
            pair_field(&pos[3 * t], &pos[3 * j], q[species[j]], species[j] != species[t], eps2,
                       E, &phi);
        }
        E_out[3 * a + 0] = E[0];
        E_out[3 * a + 1] = E[1];
        E_out[3 * a + 2] = E[2];
        phi_out[a] = phi;
    }
}

/* Direct pair energy sum_{i<j} q_i q_j / sqrt(r^2 + eps^2). */
double orc_direct_pe(int64_t n, const double* pos, const int8_t* species,
                     const double q[2], double eps)
{
    double eps2 = eps * eps, pe = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = pos[3 * i] - pos[3 * j];
            double dy = pos[3 * i + 1] - pos[3 * j + 1];
            double dz = pos[3 * i + 2] - pos[3 * j + 2];
            if (g_kelbg && species[i] != species[j]) {
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                pe += q[species[i]] * q[species[j]] *
                      (r > 0.0 ? -expm1(-r / g_lambda) / r : 1.0 / g_lambda);
            } else {
                pe += q[species[i]] * q[species[j]] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
            }
        }
    return pe;
}

/* ------------------------------------------------------------------ */
/* Sec. 3, first step (R2): a cube that encloses all particles.
 * out = {centre x, centre y, centre z, side L}. */
void orc_root_cube(int64_t n, const double* pos, double out[4])
{
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        lo[a] = n > 0 ? pos[a] : 0.0;
        hi[a] = lo[a];
    }
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = pos[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        out[a] = (lo[a] + hi[a]) * 0.5;
        if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    }
    out[3] = ext > 0.0 ? ext * (1.0 + ldexp(1.0, -20)) : 1.0;
}

/* R3: integer cell coordinates of every particle at the finest depth. */
void orc_int_coords(int64_t n, const double* pos, const double cube[4], uint32_t* k)
{
    double L = cube[3];
    double scale = (double)ORC_KMAX / L;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double lo = cube[a] - L * 0.5;
            double u = floor((pos[3 * i + a] - lo) * scale);
            uint32_t v;
            if (!(u > 0.0)) v = 0;                       /* also catches u = -0 */
            else if (u >= (double)(ORC_KMAX - 1)) v = ORC_KMAX - 1;
            else v = (uint32_t)u;
            k[3 * i + a] = v;
        }
}

/* Morton key: bit b of kx goes to key bit 3b, of ky to 3b+1, of kz to 3b+2,
 * written as a plain bit loop.  The key orders boxes depth-first with the
 * eight children of a box in octant order 0..7, octant = bx + 2 by + 4 bz. */
uint64_t orc_interleave(uint32_t kx, uint32_t ky, uint32_t kz)
{
    uint64_t key = 0;
    for (int b = 0; b < ORC_MAXDEPTH; ++b) {
        key |= (uint64_t)((kx >> b) & 1u) << (3 * b);
        key |= (uint64_t)((ky >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((kz >> b) & 1u) << (3 * b + 2);
    }
    return key;
}

void orc_keys(int64_t n, const double* pos, const double cube[4], uint64_t* keys)
{
    uint32_t* k = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)(n > 0 ? n : 1));
    orc_int_coords(n, pos, cube, k);
    for (int64_t i = 0; i < n; ++i) keys[i] = orc_interleave(k[3 * i], k[3 * i + 1], k[3 * i + 2]);
    free(k);
}

static const uint64_t* g_sort_keys; /* qsort has no context argument */
static int cmp_key_then_index(const void* pa, const void* pb)
{
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    uint64_t ka = g_sort_keys[a], kb = g_sort_keys[b];
    if (ka != kb) return ka < kb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Order of particles by (key, original index): the deterministic order that
 * any stable key sort must reproduce. */
void orc_sort_order(int64_t n, const uint64_t* keys, int64_t* order)
{
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_keys = keys;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_key_then_index);
    g_sort_keys = NULL;
}

/* ------------------------------------------------------------------ */
/* The TREE of Sec. 3 as an explicit node list in pre-order. */
typedef struct {
    int64_t n, nnodes, cap;
    int leaf_cap;
    double cube[4];
    int64_t* slot;   /* slot[s] = original particle index at tree slot s */
    uint32_t* k;     /* integer coordinates (n x 3), R3 */
    /* per node */
    int64_t *begin, *end, *next;
    int32_t *depth, *is_leaf;
    uint32_t* cell;  /* integer box coordinates at its depth (x3) */
    double *centre, *side;            /* geometric box centre (x3), side s */
    double *S0, *M, *c, *D, *Q, *delta; /* moments, R4 (c, D: x3; Q: x6) */
} orc_tree;

static int64_t new_node(orc_tree* T)
{
    if (T->nnodes == T->cap) {
        int64_t cap = T->cap ? 2 * T->cap : 1024;
#define GROW(p, ty, w) T->p = (ty*)realloc(T->p, sizeof(ty) * (size_t)(w) * (size_t)cap)
        GROW(begin, int64_t, 1); GROW(end, int64_t, 1); GROW(next, int64_t, 1);
        GROW(depth, int32_t, 1); GROW(is_leaf, int32_t, 1); GROW(cell, uint32_t, 3);
        GROW(centre, double, 3); GROW(side, double, 1); GROW(S0, double, 1);
        GROW(M, double, 1); GROW(c, double, 3); GROW(D, double, 3); GROW(Q, double, 6);
        GROW(delta, double, 1);
#undef GROW
        T->cap = cap;
    }
    return T->nnodes++;
}

/* Sec. 3: subdivide the box holding slots [b, e) into eight even boxes,
 * associate every particle with its box, and repeat until a box holds no
 * more than leaf_cap particles (or the depth cap of R3 is reached).
 * Children are appended in octant order right after their parent, so the
 * list is in pre-order; next[] is the first node after the subtree. */
static void subdivide(orc_tree* T, int64_t b, int64_t e, int d,
                      uint32_t cx, uint32_t cy, uint32_t cz, int64_t* tmp)
{
    int64_t me = new_node(T);
    T->begin[me] = b;
    T->end[me] = e;
    T->depth[me] = d;
    T->cell[3 * me] = cx;
    T->cell[3 * me + 1] = cy;
    T->cell[3 * me + 2] = cz;
    int leaf = (e - b <= T->leaf_cap) || d == ORC_MAXDEPTH;
    T->is_leaf[me] = leaf;
    if (!leaf) {
        int shift = ORC_MAXDEPTH - 1 - d; /* bit of k that picks the child */
        int64_t count[8] = {0}, start[9];
        for (int64_t s = b; s < e; ++s) {
            const uint32_t* kk = &T->k[3 * T->slot[s]];
            int oct = (int)(((kk[0] >> shift) & 1u) | (((kk[1] >> shift) & 1u) << 1) |
                            (((kk[2] >> shift) & 1u) << 2));
            count[oct]++;
        }
        start[0] = b;
        for (int o = 0; o < 8; ++o) start[o + 1] = start[o] + count[o];
        int64_t fill[8];
        for (int o = 0; o < 8; ++o) fill[o] = start[o];
        for (int64_t s = b; s < e; ++s) { /* stable partition by octant */
            const uint32_t* kk = &T->k[3 * T->slot[s]];
            int oct = (int)(((kk[0] >> shift) & 1u) | (((kk[1] >> shift) & 1u) << 1) |
                            (((kk[2] >> shift) & 1u) << 2));
            tmp[fill[oct]++] = T->slot[s];
        }
        memcpy(&T->slot[b], &tmp[b], sizeof(int64_t) * (size_t)(e - b));
        for (int o = 0; o < 8; ++o) {
            if (count[o] == 0) continue;
            subdivide(T, start[o], start[o + 1], d + 1, 2 * cx + (uint32_t)(o & 1),
                      2 * cy + (uint32_t)((o >> 1) & 1), 2 * cz + (uint32_t)((o >> 2) & 1), tmp);
        }
    }
    T->next[me] = T->nnodes;
}

/* Moments of every node straight from its own particles (R4), and the box
 * geometry used by the opening criterion (Eq. 5). */
static void node_moments(orc_tree* T, const double* pos, const int8_t* species, const double q[2])
{
    double L = T->cube[3];
    for (int64_t nd = 0; nd < T->nnodes; ++nd) {
        double s = ldexp(L, -T->depth[nd]);
        T->side[nd] = s;
        for (int a = 0; a < 3; ++a) {
            double lo = T->cube[a] - L * 0.5;
            T->centre[3 * nd + a] = lo + ((double)T->cell[3 * nd + a] + 0.5) * s;
        }
        double S0 = 0.0, M = 0.0, w[3] = {0, 0, 0};
        for (int64_t sl = T->begin[nd]; sl < T->end[nd]; ++sl) {
            int64_t j = T->slot[sl];
            double qj = q[species[j]];
            S0 += fabs(qj);
            M += qj;
            for (int a = 0; a < 3; ++a) w[a] += fabs(qj) * pos[3 * j + a];
        }
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = S0 > 0.0 ? w[a] / S0 : T->centre[3 * nd + a];
        double D[3] = {0, 0, 0}, Q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t sl = T->begin[nd]; sl < T->end[nd]; ++sl) {
            int64_t j = T->slot[sl];
            double qj = q[species[j]];
            double y[3];
            for (int a = 0; a < 3; ++a) y[a] = pos[3 * j + a] - c[a];
            for (int a = 0; a < 3; ++a) D[a] += qj * y[a];
            Q[0] += qj * y[0] * y[0]; /* xx */
            Q[1] += qj * y[0] * y[1]; /* xy */
            Q[2] += qj * y[0] * y[2]; /* xz */
            Q[3] += qj * y[1] * y[1]; /* yy */
            Q[4] += qj * y[1] * y[2]; /* yz */
            Q[5] += qj * y[2] * y[2]; /* zz */
        }
        T->S0[nd] = S0;
        T->M[nd] = M;
        for (int a = 0; a < 3; ++a) {
            T->c[3 * nd + a] = c[a];
            T->D[3 * nd + a] = D[a];
        }
        for (int a = 0; a < 6; ++a) T->Q[6 * nd + a] = Q[a];
        double ex = c[0] - T->centre[3 * nd];
        double ey = c[1] - T->centre[3 * nd + 1];
        double ez = c[2] - T->centre[3 * nd + 2];
        T->delta[nd] = sqrt(ex * ex + ey * ey + ez * ez);
    }
}

orc_tree* orc_tree_build(int64_t n, const double* pos, const int8_t* species,
                         const double q[2], int leaf_cap)
{
    orc_tree* T = (orc_tree*)calloc(1, sizeof(orc_tree));
    T->n = n;
    T->leaf_cap = leaf_cap < 1 ? 1 : leaf_cap;
    orc_root_cube(n, pos, T->cube);
    size_t nn = (size_t)(n > 0 ? n : 1);
    T->k = (uint32_t*)malloc(sizeof(uint32_t) * 3 * nn);
    orc_int_coords(n, pos, T->cube, T->k);
    T->slot = (int64_t*)malloc(sizeof(int64_t) * nn);
    for (int64_t i = 0; i < n; ++i) T->slot[i] = i;
    if (n > 0) {
        int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * nn);
        subdivide(T, 0, n, 0, 0, 0, 0, tmp);
        free(tmp);
        node_moments(T, pos, species, q);
    }
    return T;
}

void orc_tree_free(orc_tree* T)
{
    if (!T) return;
    free(T->slot); free(T->k); free(T->begin); free(T->end); free(T->next);
    free(T->depth); free(T->is_leaf); free(T->cell); free(T->centre); free(T->side);
    free(T->S0); free(T->M); free(T->c); free(T->D); free(T->Q); free(T->delta);
    free(T);
}

int64_t orc_tree_nnodes(const orc_tree* T) { return T->nnodes; }
void orc_tree_cube(const orc_tree* T, double out[4]) { memcpy(out, T->cube, sizeof(double) * 4); }

/* Copy the node table out.  topo: n_nodes x 5 int64 {begin, end, next,
 * depth, is_leaf}; cell: n_nodes x 3 uint32; geom: n_nodes x 20 double
 * {centre[3], side, S0, M, c[3], D[3], Q[6] (xx xy xz yy yz zz), delta};
 * slot: tree slot -> original index (n). Any pointer may be NULL. */
void orc_tree_export(const orc_tree* T, int64_t* topo, uint32_t* cell, double* geom, int64_t* slot)
{
    for (int64_t i = 0; i < T->nnodes; ++i) {
        if (topo) {
            topo[5 * i + 0] = T->begin[i];
            topo[5 * i + 1] = T->end[i];
            topo[5 * i + 2] = T->next[i];
            topo[5 * i + 3] = T->depth[i];
            topo[5 * i + 4] = T->is_leaf[i];
        }
        if (cell)
            for (int a = 0; a < 3; ++a) cell[3 * i + a] = T->cell[3 * i + a];
        if (geom) {
            double* g = &geom[20 * i];
            for (int a = 0; a < 3; ++a) g[a] = T->centre[3 * i + a];
            g[3] = T->side[i];
            g[4] = T->S0[i];
            g[5] = T->M[i];
            for (int a = 0; a < 3; ++a) g[6 + a] = T->c[3 * i + a];
            for (int a = 0; a < 3; ++a) g[9 + a] = T->D[3 * i + a];
            for (int a = 0; a < 6; ++a) g[12 + a] = T->Q[6 * i + a];
            g[18] = T->delta[i];
            g[19] = 0.0;
        }
    }
    if (slot) memcpy(slot, T->slot, sizeof(int64_t) * (size_t)T->n);
}

/* ------------------------------------------------------------------ */
/* R6: multipole of one node on a target at xt.  With R = xt - c,
 * g = (R.R + eps^2)^(-1/2), the potential of the node is
 *   phi = M g + (D.R) g^3 + (1/2)(3 R.Q.R g^5 - tr(Q) g^3)
 * and the field (minus its gradient) is
 *   E = M R g^3 - D g^3 + 3 (D.R) R g^5 - 3 (Q R) g^5
 *       + (15/2)(R.Q.R) R g^7 - (3/2) tr(Q) R g^5.
 * term_mask bit 0 / 1 / 2 keeps the monopole / dipole / quadrupole terms
 * (tests drop a term here to show that the pins catch it). */
static void multipole_field(const orc_tree* T, int64_t nd, const double xt[3], double eps2,
                            int term_mask, double E[3], double* phi)
{
    const double* c = &T->c[3 * nd];
    const double* D = &T->D[3 * nd];
    const double* Q = &T->Q[6 * nd];
    double M = T->M[nd];
    double R[3] = {xt[0] - c[0], xt[1] - c[1], xt[2] - c[2]};
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + eps2;
    double g = 1.0 / sqrt(r2);
    double g3 = g * g * g, g5 = g3 * g * g, g7 = g5 * g * g;
    if (term_mask & 1) {
        for (int a = 0; a < 3; ++a) E[a] += M * R[a] * g3;
        *phi += M * g;
    }
    if (term_mask & 2) {
        double DR = D[0] * R[0] + D[1] * R[1] + D[2] * R[2];
        for (int a = 0; a < 3; ++a) E[a] += -D[a] * g3 + 3.0 * DR * R[a] * g5;
        *phi += DR * g3;
    }
    if (term_mask & 4) {
        double QR[3];
        QR[0] = Q[0] * R[0] + Q[1] * R[1] + Q[2] * R[2];
        QR[1] = Q[1] * R[0] + Q[3] * R[1] + Q[4] * R[2];
        QR[2] = Q[2] * R[0] + Q[4] * R[1] + Q[5] * R[2];
        double RQR = R[0] * QR[0] + R[1] * QR[1] + R[2] * QR[2];
        double trQ = Q[0] + Q[3] + Q[5];
        for (int a = 0; a < 3; ++a)
            E[a] += -3.0 * QR[a] * g5 + 7.5 * RQR * R[a] * g7 - 1.5 * trQ * R[a] * g5;
        *phi += 0.5 * (3.0 * RQR * g5 - trQ * g3);
    }
}

typedef struct {
    const orc_tree* T;
    const double* pos;
    const int8_t* species;
    const double* q;
    double inv_theta_valid; /* 1 when theta > 0 */
    double theta, eps2;
    int term_mask;
} walk_args;

/* Sec. 3 particle-tree interaction: visit nodes from the root in pre-order,
 * children in octant order; accept a node by Eq. 5 (R5) and apply its
 * multipole, otherwise open it; an opened leaf is summed directly. */
static void walk(const walk_args* W, int64_t nd, int64_t t, const double xt[3],
                 double E[3], double* phi, int64_t* np2p, int64_t* nm2p)
{
    const orc_tree* T = W->T;
    if (W->inv_theta_valid > 0.0) {
        double rcrit = T->side[nd] / W->theta + T->delta[nd];
        double dx = xt[0] - T->c[3 * nd];
        double dy = xt[1] - T->c[3 * nd + 1];
        double dz = xt[2] - T->c[3 * nd + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (rcrit * rcrit < d2) {
            multipole_field(T, nd, xt, W->eps2, W->term_mask, E, phi);
            (*nm2p)++;
            return;
        }
    }
    if (T->is_leaf[nd]) {
        for (int64_t sl = T->begin[nd]; sl < T->end[nd]; ++sl) {
            int64_t j = T->slot[sl];
            if (j == t) continue;
            pair_field(xt, &W->pos[3 * j], W->q[W->species[j]], W->species[j] != W->species[t],
                       W->eps2, E, phi);
            (*np2p)++;
        }
        return;
    }
    for (int64_t ch = nd + 1; ch < T->next[nd]; ch = T->next[ch])
        walk(W, ch, t, xt, E, phi, np2p, nm2p);
}

/* Tree field and potential on targets tidx[0..nt) (all when NULL).
 * Outputs are per listed target; counts are optional. */
void orc_tree_force(const orc_tree* T, const double* pos, const int8_t* species,
                    const double q[2], double theta, double eps, const int64_t* tidx,
                    int64_t nt, double* E_out, double* phi_out, int64_t* np2p_out,
                    int64_t* nm2p_out, int nthreads, int term_mask)
{
    walk_args W;
    W.T = T;
    W.pos = pos;
    W.species = species;
    W.q = q;
    W.theta = theta;
    W.inv_theta_valid = theta > 0.0 ? 1.0 : 0.0;
    W.eps2 = eps * eps;
    W.term_mask = term_mask;
    if (!tidx) nt = T->n;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t a = 0; a < nt; ++a) {
        int64_t t = tidx ? tidx[a] : a;
        double E[3] = {0.0, 0.0, 0.0}, phi = 0.0;
        int64_t np = 0, nm = 0;
        if (T->nnodes > 0) walk(&W, 0, t, &pos[3 * t], E, &phi, &np, &nm);
        for (int c = 0; c < 3; ++c) E_out[3 * a + c] = E[c];
        phi_out[a] = phi;
        if (np2p_out) np2p_out[a] = np;
        if (nm2p_out) nm2p_out[a] = nm;
    }
}

/* ------------------------------------------------------------------ */
/* Acceleration of the particles whose mask entry is set: a = q_t E / m_t. */
static void accel(int64_t n, const double* pos, const int8_t* species, const double q[2],
                  const double m[2], double theta, double eps, int leaf_cap, int use_direct,
                  int only_electrons, double* acc, int nthreads)
{
    int64_t* tl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nt = 0;
    for (int64_t i = 0; i < n; ++i)
        if (!only_electrons || species[i] == 1) tl[nt++] = i;
    double* E = (double*)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    double* phi = (double*)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    if (use_direct) {
        orc_direct(n, pos, species, q, eps, tl, nt, E, phi, nthreads);
    } else {
        orc_tree* T = orc_tree_build(n, pos, species, q, leaf_cap);
        orc_tree_force(T, pos, species, q, theta, eps, tl, nt, E, phi, NULL, NULL, nthreads, 7);
        orc_tree_free(T);
    }
    for (int64_t a = 0; a < nt; ++a) {
        int64_t t = tl[a];
        double qm = q[species[t]] / m[species[t]];
        for (int c = 0; c < 3; ++c) acc[3 * t + c] = qm * E[3 * a + c];
    }
    free(tl);
    free(E);
    free(phi);
}

/* Split-step velocity Verlet (Sec. 2, velocity Verlet; the electron/ion
 * time-scale split motivates the substeps).  One block of k electron
 * substeps with dt_i = k dt_e:
 *   ions:      v += (dt_i/2) a
 *   k times:   electrons v += (dt_e/2) a;  all x += dt_e v;
 *              new tree; a for electrons (for all particles on substep k);
 *              electrons v += (dt_e/2) a
 *   ions:      v += (dt_i/2) a
 * With k = 1 this is plain velocity Verlet.  acc holds the accelerations of
 * the current positions on entry (computed here first when acc_valid = 0)
 * and on exit. */
void orc_run(int64_t n, double* pos, double* vel, const int8_t* species, const double q[2],
             const double m[2], double dt_e, int k, int64_t nblocks, double theta, double eps,
             int leaf_cap, int use_direct, double* acc, int acc_valid, int nthreads)
{
    if (!acc_valid)
        accel(n, pos, species, q, m, theta, eps, leaf_cap, use_direct, 0, acc, nthreads);
    double dt_i = k * dt_e;
    for (int64_t blk = 0; blk < nblocks; ++blk) {
        for (int64_t i = 0; i < n; ++i)
            if (species[i] == 0)
                for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt_i * acc[3 * i + c];
        for (int s = 1; s <= k; ++s) {
            for (int64_t i = 0; i < n; ++i)
                if (species[i] == 1)
                    for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt_e * acc[3 * i + c];
            for (int64_t i = 0; i < 3 * n; ++i) pos[i] += dt_e * vel[i];
            accel(n, pos, species, q, m, theta, eps, leaf_cap, use_direct, s < k, acc, nthreads);
            for (int64_t i = 0; i < n; ++i)
                if (species[i] == 1)
                    for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt_e * acc[3 * i + c];
        }
        for (int64_t i = 0; i < n; ++i)
            if (species[i] == 0)
                for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt_i * acc[3 * i + c];
    }
}

/* Sec. 5 observables.  out = {KE_ion, KE_electron, PE, E = KE + PE, |P|}.
 * PE = (1/2) sum_t q_t phi_t with the tree potential (or the direct pair sum
 * when use_direct).  Temperature of species s is 2 KE_s / (3 N_s). */
void orc_energy(int64_t n, const double* pos, const double* vel, const int8_t* species,
                const double q[2], const double m[2], double theta, double eps, int leaf_cap,
                int use_direct, double out[5], int nthreads)
{
    double ke[2] = {0.0, 0.0}, P[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        int s = species[i];
        double v2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            v2 += vel[3 * i + c] * vel[3 * i + c];
            P[c] += m[s] * vel[3 * i + c];
        }
        ke[s] += 0.5 * m[s] * v2;
    }
    double pe = 0.0;
    if (use_direct) {
        pe = orc_direct_pe(n, pos, species, q, eps);
    } else {
        double* E = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
        double* phi = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        orc_tree* T = orc_tree_build(n, pos, species, q, leaf_cap);
        orc_tree_force(T, pos, species, q, theta, eps, NULL, n, E, phi, NULL, NULL, nthreads, 7);
        orc_tree_free(T);
        for (int64_t i = 0; i < n; ++i) pe += 0.5 * q[species[i]] * phi[i];
        free(E);
        free(phi);
    }
    out[0] = ke[0];
    out[1] = ke[1];
    out[2] = pe;
    out[3] = ke[0] + ke[1] + pe;
    out[4] = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
}

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Multipole (R6) of one box holding all n particles, evaluated at xt, next to
 * nothing else: the tree is built with leaf_cap = n so that the root is the
 * only node and its moments come from the same code as every other node. */
void orc_cluster_multipole(int64_t n, const double* pos, const int8_t* species,
                           const double q[2], double eps, const double xt[3], int term_mask,
                           double E[3], double* phi)
{
    orc_tree* T = orc_tree_build(n, pos, species, q, (int)(n > 0 ? n : 1));
    E[0] = E[1] = E[2] = 0.0;
    *phi = 0.0;
    if (T->nnodes > 0) multipole_field(T, 0, xt, eps * eps, term_mask, E, phi);
    orc_tree_free(T);
}

/* ------------------------------------------------------------------ */
/* Adjoint of the TREE force (the derivative the split-step push needs to carry
 * gradients back through a run).  For a cotangent lambda (n x 3, per original
 * index) it returns mu = (d a / d x)^T lambda, a = q E / m, with the tree held
 * fixed (which boxes each target opens or accepts does not move under an
 * infinitesimal displacement).  Every piece is the exact derivative of what
 * orc_tree_force computes:
 *   - a direct pair: J(r) = d/dr [r g^3] = g^3 I - 3 g^5 r r^T, on the target
 *     side and, with the opposite sign, on the source side;
 *   - an accepted box, target side: the field gradient of the expansion,
 *     -(M grad grad g - D . grad^3 g + 1/2 Q : grad^4 g);
 *   - an accepted box, source side: through D and Q at fixed centre
 *     (q_s [alpha - Gamma y_s]) and through the centre c = sum |q| x / S0 that
 *     the expansion is taken about (|q_s| / S0 kappa), where, with
 *     w = q_t lambda_t / m_t summed over the targets that accept the box,
 *     alpha = grad grad g w, Gamma_ec = w_a d_aec g, kappa = 1/2 grad^4 g[w, ., Q].
 * Derivatives of g = (R.R + eps^2)^(-1/2):
 *   d_ab g   = 3 R_a R_b g^5 - d_ab g^3
 *   d_abc g  = -15 R_a R_b R_c g^7 + 3 (d_ab R_c + d_ac R_b + d_bc R_a) g^5
 *   d_abcd g = 105 R_a R_b R_c R_d g^9 - 15 (six d_xy R R terms) g^7
 *              + 3 (d_ab d_cd + d_ac d_bd + d_ad d_bc) g^5 */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Q (xx xy xz yy yz zz) times v */
static void qmul(const double* Q, const double* v, double out[3])
{
    out[0] = Q[0] * v[0] + Q[1] * v[1] + Q[2] * v[2];
    out[1] = Q[1] * v[0] + Q[3] * v[1] + Q[4] * v[2];
    out[2] = Q[2] * v[0] + Q[4] * v[1] + Q[5] * v[2];
}

/* sum_bcd v_b Q_cd d_abcd g, free index a */
static void t4(const double R[3], const double v[3], const double* Q, double g, double out[3])
{
    double g2 = g * g, g5 = g2 * g2 * g, g7 = g5 * g2, g9 = g7 * g2;
    double QR[3], Qv[3];
    qmul(Q, R, QR);
    qmul(Q, v, Qv);
    double RQR = dot3(R, QR), Rv = dot3(R, v), vQR = dot3(v, QR), trQ = Q[0] + Q[3] + Q[5];
    for (int a = 0; a < 3; ++a)
        out[a] = 105.0 * R[a] * Rv * RQR * g9
                 - 15.0 * g7 * (v[a] * RQR + 2.0 * Rv * QR[a] + 2.0 * R[a] * vQR + R[a] * Rv * trQ)
                 + 3.0 * g5 * (v[a] * trQ + 2.0 * Qv[a]);
}

typedef struct {
    const orc_tree* T;
    const double* pos;
    const int8_t* species;
    const double *q, *m;
    double theta, eps2;
    double *alpha, *gam, *kap, *mu;
} adj_args;

static void walk_adj(const adj_args* A, int64_t nd, int64_t t, const double xt[3], const double lam[3],
                     const double w[3], double qt_over_mt, double mu_t[3])
{
    const orc_tree* T = A->T;
    if (A->theta > 0.0) {
        double rcrit = T->side[nd] / A->theta + T->delta[nd];
        double dx = xt[0] - T->c[3 * nd];
        double dy = xt[1] - T->c[3 * nd + 1];
        double dz = xt[2] - T->c[3 * nd + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (rcrit * rcrit < d2) {
            const double* D = &T->D[3 * nd];
            const double* Q = &T->Q[6 * nd];
            double M = T->M[nd];
            double R[3] = {dx, dy, dz};
            double g = 1.0 / sqrt(d2 + A->eps2);
            double g2 = g * g, g3 = g2 * g, g5 = g3 * g2, g7 = g5 * g2;
            /* target side: -(M grad grad g lam - sum_bc lam_b D_c d_abc g + 1/2 T4(lam)) */
            double Rl = dot3(R, lam), RD = dot3(R, D), lD = dot3(lam, D);
            double T4l[3];
            t4(R, lam, Q, g, T4l);
            for (int a = 0; a < 3; ++a) {
                double hess = M * (3.0 * R[a] * Rl * g5 - lam[a] * g3);
                double dterm = -15.0 * R[a] * Rl * RD * g7 + 3.0 * (lam[a] * RD + D[a] * Rl + R[a] * lD) * g5;
                mu_t[a] += qt_over_mt * -(hess - dterm + 0.5 * T4l[a]);
            }
            /* source side accumulators of the box */
            double Rw = dot3(R, w);
            double T4w[3];
            t4(R, w, Q, g, T4w);
            for (int a = 0; a < 3; ++a) {
                A->alpha[3 * nd + a] += 3.0 * R[a] * Rw * g5 - w[a] * g3;
                A->kap[3 * nd + a] += 0.5 * T4w[a];
            }
            const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
            for (int k = 0; k < 6; ++k) {
                int e = ia[k], c = ib[k];
                A->gam[6 * nd + k] += -15.0 * Rw * R[e] * R[c] * g7 +
                                      3.0 * (w[e] * R[c] + w[c] * R[e] + (e == c ? Rw : 0.0)) * g5;
            }
            return;
        }
    }
    if (T->is_leaf[nd]) {
        for (int64_t sl = T->begin[nd]; sl < T->end[nd]; ++sl) {
            int64_t j = T->slot[sl];
            if (j == t) continue;
            double qj = A->q[A->species[j]];
            double r[3] = {xt[0] - A->pos[3 * j], xt[1] - A->pos[3 * j + 1], xt[2] - A->pos[3 * j + 2]};
            double g = 1.0 / sqrt(dot3(r, r) + A->eps2);
            double g3 = g * g * g, g5 = g3 * g * g;
            double rl = dot3(r, lam), rw = dot3(r, w);
            for (int a = 0; a < 3; ++a) {
                mu_t[a] += qt_over_mt * qj * (lam[a] * g3 - 3.0 * r[a] * rl * g5);
                A->mu[3 * j + a] -= qj * (w[a] * g3 - 3.0 * r[a] * rw * g5);
            }
        }
        return;
    }
    for (int64_t ch = nd + 1; ch < T->next[nd]; ch = T->next[ch])
        walk_adj(A, ch, t, xt, lam, w, qt_over_mt, mu_t);
}

void orc_tree_force_adjoint(const orc_tree* T, const double* pos, const int8_t* species,
                            const double q[2], const double m[2], double theta, double eps,
                            const double* lam, double* mu)
{
    int64_t n = T->n, nn = T->nnodes;
    adj_args A;
    A.T = T;
    A.pos = pos;
    A.species = species;
    A.q = q;
    A.m = m;
    A.theta = theta;
    A.eps2 = eps * eps;
    A.alpha = (double*)calloc((size_t)(3 * nn + 1), sizeof(double));
    A.gam = (double*)calloc((size_t)(6 * nn + 1), sizeof(double));
    A.kap = (double*)calloc((size_t)(3 * nn + 1), sizeof(double));
    A.mu = mu;
    memset(mu, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t t = 0; t < n; ++t) {
        const double* l = &lam[3 * t];
        if (l[0] == 0.0 && l[1] == 0.0 && l[2] == 0.0) continue;
        double qm = q[species[t]] / m[species[t]];
        double w[3] = {qm * l[0], qm * l[1], qm * l[2]};
        double mu_t[3] = {0.0, 0.0, 0.0};
        if (nn > 0) walk_adj(&A, 0, t, &pos[3 * t], l, w, qm, mu_t);
        for (int a = 0; a < 3; ++a) mu[3 * t + a] += mu_t[a];
    }
    /* push the box accumulators down to the particles of each box */
    for (int64_t nd = 0; nd < nn; ++nd) {
        const double* c = &T->c[3 * nd];
        const double* G = &A.gam[6 * nd];
        for (int64_t sl = T->begin[nd]; sl < T->end[nd]; ++sl) {
            int64_t s = T->slot[sl];
            double qs = q[species[s]];
            double y[3] = {pos[3 * s] - c[0], pos[3 * s + 1] - c[1], pos[3 * s + 2] - c[2]};
            double Gy[3];
            qmul(G, y, Gy);
            double cw = T->S0[nd] > 0.0 ? fabs(qs) / T->S0[nd] : 0.0;
            for (int a = 0; a < 3; ++a)
                mu[3 * s + a] += qs * (A.alpha[3 * nd + a] - Gy[a]) + cw * A.kap[3 * nd + a];
        }
    }
    free(A.alpha);
    free(A.gam);
    free(A.kap);
}

/* Adjoint of the direct sum (the same pair derivative over all pairs). */
void orc_direct_force_adjoint(int64_t n, const double* pos, const int8_t* species, const double q[2],
                              const double m[2], double eps, const double* lam, double* mu)
{
    double eps2 = eps * eps;
    memset(mu, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t t = 0; t < n; ++t) {
        const double* l = &lam[3 * t];
        double qm = q[species[t]] / m[species[t]];
        double w[3] = {qm * l[0], qm * l[1], qm * l[2]};
        for (int64_t j = 0; j < n; ++j) {
            if (j == t) continue;
            double qj = q[species[j]];
            double r[3] = {pos[3 * t] - pos[3 * j], pos[3 * t + 1] - pos[3 * j + 1], pos[3 * t + 2] - pos[3 * j + 2]};
            double g = 1.0 / sqrt(dot3(r, r) + eps2);
            double g3 = g * g * g, g5 = g3 * g * g;
            double rl = dot3(r, l), rw = dot3(r, w);
            for (int a = 0; a < 3; ++a) {
                mu[3 * t + a] += qm * qj * (l[a] * g3 - 3.0 * r[a] * rl * g5);
                mu[3 * j + a] -= qj * (w[a] * g3 - 3.0 * r[a] * rw * g5);
            }
        }
    }
}

static void force_adjoint_at(int64_t n, const double* x, const int8_t* species, const double q[2],
                             const double m[2], double theta, double eps, int leaf_cap,
                             int use_direct, const double* lam, double* mu)
{
    if (use_direct) {
        orc_direct_force_adjoint(n, x, species, q, m, eps, lam, mu);
    } else {
        orc_tree* T = orc_tree_build(n, x, species, q, leaf_cap);
        orc_tree_force_adjoint(T, x, species, q, m, theta, eps, lam, mu);
        orc_tree_free(T);
    }
}

/* Gradient of L = electron kinetic energy after nblocks blocks of orc_run (from
 * (pos, vel) with no stored accelerations) with respect to the initial
 * positions and velocities: the push run forward once, every substep position
 * kept, then the exact reverse of each kick and drift (velocity Verlet is
 * linear in v, and each kick v += h a(x) sends lambda_x += h (da/dx)^T lambda_v
 * on the kicked species' rows).  Returns L. */
double orc_run_adjoint_ke_e(int64_t n, const double* pos, const double* vel, const int8_t* species,
                            const double q[2], const double m[2], double dt_e, int k,
                            int64_t nblocks, double theta, double eps, int leaf_cap, int use_direct,
                            double* grad_x, double* grad_v, int nthreads)
{
    int64_t S = nblocks * k;
    size_t nb3 = 3 * (size_t)n;
    double* X = (double*)malloc(sizeof(double) * nb3 * (size_t)(S + 1));
    double* v = (double*)malloc(sizeof(double) * nb3);
    double* acc = (double*)malloc(sizeof(double) * nb3);
    memcpy(X, pos, sizeof(double) * nb3);
    memcpy(v, vel, sizeof(double) * nb3);
    accel(n, X, species, q, m, theta, eps, leaf_cap, use_direct, 0, acc, nthreads);
    double dt_i = k * dt_e;
    for (int64_t b = 0; b < nblocks; ++b) {
        for (int64_t i = 0; i < n; ++i)
            if (species[i] == 0)
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt_i * acc[3 * i + c];
        for (int s = 1; s <= k; ++s) {
            int64_t g = b * k + s;
            double* xp = X + nb3 * (size_t)(g - 1);
            double* xg = X + nb3 * (size_t)g;
            for (int64_t i = 0; i < n; ++i)
                if (species[i] == 1)
                    for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt_e * acc[3 * i + c];
            for (size_t i = 0; i < nb3; ++i) xg[i] = xp[i] + dt_e * v[i];
            accel(n, xg, species, q, m, theta, eps, leaf_cap, use_direct, s < k, acc, nthreads);
            for (int64_t i = 0; i < n; ++i)
                if (species[i] == 1)
                    for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt_e * acc[3 * i + c];
        }
        for (int64_t i = 0; i < n; ++i)
            if (species[i] == 0)
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt_i * acc[3 * i + c];
    }
    double L = 0.0;
    double* lx = grad_x;
    double* lv = grad_v;
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            lx[3 * i + c] = 0.0;
            lv[3 * i + c] = species[i] == 1 ? m[1] * v[3 * i + c] : 0.0;
            if (species[i] == 1) L += 0.5 * m[1] * v[3 * i + c] * v[3 * i + c];
        }
    double* lam = (double*)malloc(sizeof(double) * nb3);
    double* mu = (double*)malloc(sizeof(double) * nb3);
#define KICK_ADJ(XPOS, H, SPEC)                                                                \
    do {                                                                                       \
        for (int64_t i = 0; i < n; ++i)                                                        \
            for (int c = 0; c < 3; ++c)                                                        \
                lam[3 * i + c] = species[i] == (SPEC) ? (H) * lv[3 * i + c] : 0.0;             \
        force_adjoint_at(n, XPOS, species, q, m, theta, eps, leaf_cap, use_direct, lam, mu);   \
        for (size_t i = 0; i < nb3; ++i) lx[i] += mu[i];                                       \
    } while (0)
    for (int64_t b = nblocks - 1; b >= 0; --b) {
        KICK_ADJ(X + nb3 * (size_t)((b + 1) * k), 0.5 * dt_i, 0);
        for (int s = k; s >= 1; --s) {
            int64_t g = b * k + s;
            KICK_ADJ(X + nb3 * (size_t)g, 0.5 * dt_e, 1);
            for (size_t i = 0; i < nb3; ++i) lv[i] += dt_e * lx[i];
            KICK_ADJ(X + nb3 * (size_t)(g - 1), 0.5 * dt_e, 1);
        }
        KICK_ADJ(X + nb3 * (size_t)(b * k), 0.5 * dt_i, 0);
    }
#undef KICK_ADJ
    free(lam);
    free(mu);
    free(X);
    free(v);
    free(acc);
    return L;
}
