/* A plain C client of libucp.so: reads a cloud (N, then N lines of x y z vx vy vz
 * species), builds a context through the C ABI only, and writes the tree force,
 * the state after a few substeps and the energy.  Used by test_gpu_c_abi.py. */
#include <stdio.h>
#include <stdlib.h>

#include "ucp.h"

static int check(int rc, ucp_ctx* ctx, const char* what)
{
    if (rc != UCP_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, ucp_strerror(rc), ctx ? ucp_last_error(ctx) : "");
        return 1;
    }
    return 0;
}

int main(int argc, char** argv)
{
    if (argc != 4) {
        fprintf(stderr, "usage: %s in.txt out.txt precision\n", argv[0]);
        return 2;
    }
    FILE* in = fopen(argv[1], "r");
    if (!in) return 2;
    long long n = 0;
    if (fscanf(in, "%lld", &n) != 1 || n < 1) return 2;
    double* pos = malloc(sizeof(double) * 3 * n);
    double* vel = malloc(sizeof(double) * 3 * n);
    int8_t* sp = malloc((size_t)n);
    double* acc = malloc(sizeof(double) * 3 * n);
    double* phi = malloc(sizeof(double) * n);
    for (long long i = 0; i < n; ++i) {
        int s = 0;
        if (fscanf(in, "%lf %lf %lf %lf %lf %lf %d", &pos[3 * i], &pos[3 * i + 1], &pos[3 * i + 2],
                   &vel[3 * i], &vel[3 * i + 1], &vel[3 * i + 2], &s) != 7)
            return 2;
        sp[i] = (int8_t)s;
    }
    fclose(in);

    ucp_params p = {0};
    p.n = n;
    p.leaf_cap = 16;
    p.precision = atoi(argv[3]);
    p.q[UCP_ION] = 1.0;
    p.q[UCP_ELECTRON] = -1.0;
    p.m[UCP_ION] = 1000.0;
    p.m[UCP_ELECTRON] = 1.0;
    p.cuda_stream = NULL;
    p.potential = UCP_POT_PLUMMER;
    ucp_ctx* ctx = NULL;
    double e[6];
    if (check(ucp_create(&ctx, &p), NULL, "ucp_create") ||
        check(ucp_set_state(ctx, pos, vel, sp, 0), ctx, "ucp_set_state") ||
        check(ucp_tree_force(ctx, 0.5, 0.01, acc, phi, 0), ctx, "ucp_tree_force"))
        return 1;
    FILE* out = fopen(argv[2], "w");
    for (long long i = 0; i < n; ++i)
        fprintf(out, "%.17g %.17g %.17g %.17g\n", acc[3 * i], acc[3 * i + 1], acc[3 * i + 2], phi[i]);
    if (check(ucp_step(ctx, 1e-3, 5, 10, 0.5, 0.01), ctx, "ucp_step") ||
        check(ucp_get_state(ctx, pos, vel, 0), ctx, "ucp_get_state") ||
        check(ucp_energy(ctx, 0.5, 0.01, e), ctx, "ucp_energy"))
        return 1;
    for (long long i = 0; i < n; ++i)
        fprintf(out, "%.17g %.17g %.17g %.17g %.17g %.17g\n", pos[3 * i], pos[3 * i + 1],
                pos[3 * i + 2], vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]);
    fprintf(out, "%.17g %.17g %.17g %.17g %.17g %.17g\n", e[0], e[1], e[2], e[3], e[4], e[5]);
    fclose(out);
    ucp_destroy(ctx);
    free(pos);
    free(vel);
    free(sp);
    free(acc);
    free(phi);
    return 0;
}
