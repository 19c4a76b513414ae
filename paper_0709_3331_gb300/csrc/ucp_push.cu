// ucp_push.cu -- velocity Verlet kicks and drifts (Sec. 2 of arXiv 0709.3331),
// the key-order permutation of the particle state, target selection, energy
// and momentum reductions (Sec. 5), and layout conversions at the boundary.
#include "ucp_internal.cuh"

#include <math.h>

namespace ucp {

namespace {

constexpr int kT = 256;

__global__ void k_permute(const unsigned int* __restrict__ perm, int n,
                          const double* __restrict__ s0, const double* __restrict__ s1,
                          const double* __restrict__ s2, const double* __restrict__ s3,
                          const double* __restrict__ s4, const double* __restrict__ s5,
                          double* __restrict__ d0, double* __restrict__ d1, double* __restrict__ d2,
                          double* __restrict__ d3, double* __restrict__ d4, double* __restrict__ d5,
                          const int8_t* __restrict__ spi, int8_t* __restrict__ spo,
                          const unsigned int* __restrict__ idi, unsigned int* __restrict__ ido)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned int p = perm[i];
    d0[i] = s0[p];
    d1[i] = s1[p];
    d2[i] = s2[p];
    d3[i] = s3[p];
    d4[i] = s4[p];
    d5[i] = s5[p];
    spo[i] = spi[p];
    ido[i] = idi[p];
}

__global__ void k_kick(double* __restrict__ vx, double* __restrict__ vy, double* __restrict__ vz,
                       const double* __restrict__ ax, const double* __restrict__ ay,
                       const double* __restrict__ az, const int8_t* __restrict__ sp, int species,
                       double h, int n, int times)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || sp[i] != species) return;
    double ux = vx[i], uy = vy[i], uz = vz[i];
    double gx = ax[i], gy = ay[i], gz = az[i];
    // consecutive half kicks, each rounded on its own, each one fused
    // multiply-add (one FP64 operation per component: GB300's FP64 rate is 1/64
    // of FP32); written out so that every kernel that kicks gives the same bits
    for (int k = 0; k < times; ++k) {
        ux = __fma_rn(h, gx, ux);
        uy = __fma_rn(h, gy, uy);
        uz = __fma_rn(h, gz, uz);
    }
    vx[i] = ux;
    vy[i] = uy;
    vz[i] = uz;
}

__global__ void k_drift(double* __restrict__ x, double* __restrict__ y, double* __restrict__ z,
                        const double* __restrict__ vx, const double* __restrict__ vy,
                        const double* __restrict__ vz, double dt, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = __fma_rn(dt, vx[i], x[i]);  // one rounding, as the kicks
    y[i] = __fma_rn(dt, vy[i], y[i]);
    z[i] = __fma_rn(dt, vz[i], z[i]);
}

// Deterministic two-level reduction: fixed per-thread strides, fixed tree in
// the block, partials summed in block order by one thread.
// out6 = {KE_ion, KE_electron, PE, px, py, pz}
__global__ void k_energy_partial(const double* __restrict__ vx, const double* __restrict__ vy,
                                 const double* __restrict__ vz, const double* __restrict__ phi,
                                 const int8_t* __restrict__ sp, const double* __restrict__ qsp,
                                 const double* __restrict__ msp, int n, double* __restrict__ part)
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int s = sp[i];
        double m = msp[s];
        double ux = vx[i], uy = vy[i], uz = vz[i];
        double ke = 0.5 * m * (ux * ux + uy * uy + uz * uz);
        acc[s] += ke;
        acc[2] += 0.5 * qsp[s] * phi[i];
        acc[3] += m * ux;
        acc[4] += m * uy;
        acc[5] += m * uz;
    }
    __shared__ double sh[kT][6];
    for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + st][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = sh[0][k];
}

// Per-cloud observables, one block per cloud over its segment (fixed order):
// out[6 c ..] = {KE_ion, KE_electron, PE, px, py, pz}
__global__ void k_energy_clouds(const double* __restrict__ vx, const double* __restrict__ vy,
                                const double* __restrict__ vz, const double* __restrict__ phi,
                                const int8_t* __restrict__ sp, const double* __restrict__ qsp,
                                const double* __restrict__ msp, const int* __restrict__ cloud_start,
                                double* __restrict__ out)
{
    const int c = blockIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = cloud_start[c] + threadIdx.x; i < cloud_start[c + 1]; i += blockDim.x) {
        int s = sp[i];
        double m = msp[s];
        double ux = vx[i], uy = vy[i], uz = vz[i];
        acc[s] += 0.5 * m * (ux * ux + uy * uy + uz * uz);
        acc[2] += 0.5 * qsp[s] * phi[i];
        acc[3] += m * ux;
        acc[4] += m * uy;
        acc[5] += m * uz;
    }
    __shared__ double sh[kT][6];
    for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + st][k];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[6 * c + threadIdx.x] = sh[0][threadIdx.x];
}

// Six warps, one per observable: lane l adds partials l, l + 32, ..., then the
// lanes are added by a fixed butterfly (a deterministic order).
__global__ void __launch_bounds__(192)
k_energy_final(const double* __restrict__ part, int nblk, double* __restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int b = lane; b < nblk; b += 32) acc += part[6 * b + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[k] = acc;
}

__global__ void k_scatter3(const double* __restrict__ ax, const double* __restrict__ ay,
                           const double* __restrict__ az, const unsigned int* __restrict__ id,
                           int n, double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned int j = id[i];
    out[3 * (size_t)j] = ax[i];
    out[3 * (size_t)j + 1] = ay[i];
    out[3 * (size_t)j + 2] = az[i];
}

__global__ void k_scatter1(const double* __restrict__ a, const unsigned int* __restrict__ id, int n,
                           double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[id[i]] = a[i];
}

__global__ void k_scatter_int(const int* __restrict__ a, const unsigned int* __restrict__ id, int n,
                              int* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[id[i]] = a[i];
}

__global__ void k_deinterleave(const double* __restrict__ aos, int n, double* __restrict__ x,
                               double* __restrict__ y, double* __restrict__ z)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = aos[3 * (size_t)i];
    y[i] = aos[3 * (size_t)i + 1];
    z[i] = aos[3 * (size_t)i + 2];
}

// flags[0] |= 1 on a non-finite position or velocity, flags[1] |= 1 on a
// species code other than 0 or 1.
__global__ void k_check_state(const double* __restrict__ pos, const double* __restrict__ vel,
                              const int8_t* __restrict__ sp, int n, int* __restrict__ flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool bad = false;
    for (int a = 0; a < 3; ++a)
        bad |= !isfinite(pos[3 * (size_t)i + a]) || !isfinite(vel[3 * (size_t)i + a]);
    if (bad) atomicOr(&flags[0], 1);
    if (sp[i] != 0 && sp[i] != 1) atomicOr(&flags[1], 1);
}

__global__ void k_iota(unsigned int* a, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (unsigned int)i;
}

inline int nb(int n) { return (n + kT - 1) / kT > 0 ? (n + kT - 1) / kT : 1; }

}  // namespace

void launch_permute(const unsigned int* perm, int n, const double* const* src6, double* const* dst6,
                    const int8_t* sp_in, int8_t* sp_out, const unsigned int* id_in,
                    unsigned int* id_out, cudaStream_t s)
{
    count_launch(1);
    k_permute<<<nb(n), kT, 0, s>>>(perm, n, src6[0], src6[1], src6[2], src6[3], src6[4], src6[5],
                                   dst6[0], dst6[1], dst6[2], dst6[3], dst6[4], dst6[5], sp_in,
                                   sp_out, id_in, id_out);
}

void launch_kick(double* vx, double* vy, double* vz, const double* ax, const double* ay,
                 const double* az, const int8_t* sp, int species, double h, int n, int times,
                 cudaStream_t s)
{
    count_launch(1);
    k_kick<<<nb(n), kT, 0, s>>>(vx, vy, vz, ax, ay, az, sp, species, h, n, times);
}

void launch_drift(double* x, double* y, double* z, const double* vx, const double* vy,
                  const double* vz, double dt, int n, cudaStream_t s)
{
    count_launch(1);
    k_drift<<<nb(n), kT, 0, s>>>(x, y, z, vx, vy, vz, dt, n);
}

void launch_energy(const double* vx, const double* vy, const double* vz, const double* phi,
                   const int8_t* sp, const double* qsp, const double* msp, int n,
                   double* partials, int nblk, double* out6, cudaStream_t s)
{
    count_launch(2);
    k_energy_partial<<<nblk, kT, 0, s>>>(vx, vy, vz, phi, sp, qsp, msp, n, partials);
    k_energy_final<<<1, 192, 0, s>>>(partials, nblk, out6);
}

void launch_energy_clouds(const double* vx, const double* vy, const double* vz, const double* phi,
                          const int8_t* sp, const double* qsp, const double* msp,
                          const int* cloud_start, int n_clouds, double* out, cudaStream_t s)
{
    count_launch(1);
    k_energy_clouds<<<n_clouds, kT, 0, s>>>(vx, vy, vz, phi, sp, qsp, msp, cloud_start, out);
}

void launch_scatter3(const double* ax, const double* ay, const double* az, const unsigned int* id,
                     int n, double* out, cudaStream_t s)
{
    count_launch(1);
    k_scatter3<<<nb(n), kT, 0, s>>>(ax, ay, az, id, n, out);
}

void launch_scatter1(const double* a, const unsigned int* id, int n, double* out, cudaStream_t s)
{
    count_launch(1);
    k_scatter1<<<nb(n), kT, 0, s>>>(a, id, n, out);
}

void launch_scatter_int(const int* a, const unsigned int* id, int n, int* out, cudaStream_t s)
{
    count_launch(1);
    k_scatter_int<<<nb(n), kT, 0, s>>>(a, id, n, out);
}

void launch_deinterleave(const double* aos, int n, double* x, double* y, double* z, cudaStream_t s)
{
    count_launch(1);
    k_deinterleave<<<nb(n), kT, 0, s>>>(aos, n, x, y, z);
}

void launch_check_state(const double* pos, const double* vel, const int8_t* sp, int n, int* flags,
                        cudaStream_t s)
{
    count_launch(1);
    k_check_state<<<nb(n), kT, 0, s>>>(pos, vel, sp, n, flags);
}

void launch_iota(unsigned int* a, int n, cudaStream_t s)
{
    count_launch(1);
    k_iota<<<nb(n), kT, 0, s>>>(a, n);
}

}  // namespace ucp
