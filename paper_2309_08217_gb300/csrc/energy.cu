// energy.cu -- conserved quantities for the diagnostics of Sect. 3.1
// (dE/E = E(t)/E0 - 1, dL/L = L(t)/L0 - 1), FP64:
//
//   E = sum m_i v_i^2 / 2 + |P|^2 / (2 M*) - sum G M* m_i / r_i - sum_{i<j} G m_i m_j / r_ij
//   L = sum m_i x_i cross v_i
//
// (the democratic-heliocentric Hamiltonian; P = sum m v).  Each thread owns
// one body i and sums its j > i pair terms with compensation; blocks reduce
// in a fixed tree order, and the host adds the block results in index order,
// so the diagnostics are reproducible.  This is off the timed path.
#include "internal.cuh"

namespace genga {

namespace {

constexpr int EN_THREADS = 256;

struct NS {
    double s = 0.0, c = 0.0;
    __device__ void add(double v) {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ double value() const { return s + c; }
};

__global__ void __launch_bounds__(EN_THREADS) energy_kernel(const double *__restrict__ x,
                                                            const double *__restrict__ y,
                                                            const double *__restrict__ z,
                                                            const double *__restrict__ vx,
                                                            const double *__restrict__ vy,
                                                            const double *__restrict__ vz,
                                                            const double *__restrict__ m, int N, double G,
                                                            double Mstar, int n_big, double *__restrict__ part) {
    __shared__ double sh[4][EN_THREADS];
    const int i = blockIdx.x * EN_THREADS + threadIdx.x;
    double e = 0.0, lx = 0.0, ly = 0.0, lz = 0.0;
    if (i < N) {
        const double xi = x[i], yi = y[i], zi = z[i], mi = m[i];
        const double ui = vx[i], vi = vy[i], wi = vz[i];
        NS pot;
        // test-particle mode 2: no potential between two test particles
        const int jend = (n_big >= 0 && i >= n_big) ? i + 1 : N;  // j > i >= n_big: both test particles
        for (int j = i + 1; j < jend; j++) {
            const double dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
            pot.add(m[j] / sqrt(dx * dx + dy * dy + dz * dz));
        }
        NS en;
        en.add(0.5 * mi * (ui * ui + vi * vi + wi * wi));
        en.add(-G * Mstar * mi / sqrt(xi * xi + yi * yi + zi * zi));
        en.add(-G * mi * pot.value());
        e = en.value();
        lx = mi * (yi * wi - zi * vi);
        ly = mi * (zi * ui - xi * wi);
        lz = mi * (xi * vi - yi * ui);
    }
    sh[0][threadIdx.x] = e;
    sh[1][threadIdx.x] = lx;
    sh[2][threadIdx.x] = ly;
    sh[3][threadIdx.x] = lz;
    __syncthreads();
    for (int w = EN_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; c++) part[4 * blockIdx.x + c] = sh[c][0];
}

}  // namespace

cudaError_t launch_energy(const genga_system &sys, const genga_params &p, genga_ctx *c, cudaStream_t s) {
    const int nb = (sys.N + EN_THREADS - 1) / EN_THREADS;
    if (nb == 0) return cudaSuccess;
    energy_kernel<<<nb, EN_THREADS, 0, s>>>(sys.x, sys.y, sys.z, sys.vx, sys.vy, sys.vz, sys.m, sys.N, p.G,
                                            p.Mstar, p.n_big, c->energy_part);
    return cudaGetLastError();
}

}  // namespace genga
