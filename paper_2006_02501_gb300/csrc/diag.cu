// Diagnostics: total energy (kinetic + softened pair potential, FP64) and
// Laplace-Runge-Lenz / eccentricity vectors (Dittmann 2020, Appendix A, Eq. A1).
#include "common.cuh"

namespace mh {

namespace {

constexpr int kDiagThreads = 256;

// Per-block partial of  sum_i m_i |v_i|^2 / 2  -  (G/2) sum_i m_i sum_{j != i} m_j / sqrt(r^2 + eps^2).
__global__ void __launch_bounds__(kDiagThreads) k_energy(int64_t N, int64_t ld, const double *m,
                                                         const double *x, const double *v,
                                                         double eps2, double G, double *partial)
{
    __shared__ double sx[3][kDiagThreads];
    __shared__ double sm[kDiagThreads];
    __shared__ double red[kDiagThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < N;
    const int64_t ic = live ? i : 0;
    const double xi = x[ic], yi = x[ld + ic], zi = x[2 * ld + ic];
    double pot = 0.0;
    for (int64_t j0 = 0; j0 < N; j0 += kDiagThreads) {
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        sx[0][threadIdx.x] = j < N ? x[j] : 0.0;
        sx[1][threadIdx.x] = j < N ? x[ld + j] : 0.0;
        sx[2][threadIdx.x] = j < N ? x[2 * ld + j] : 0.0;
        sm[threadIdx.x] = j < N ? m[j] : 0.0;
        __syncthreads();
        const int nj = (int)min((int64_t)kDiagThreads, N - j0);
        for (int jj = 0; jj < nj; ++jj) {
            if (j0 + jj == ic) continue;
            const double dx = sx[0][jj] - xi, dy = sx[1][jj] - yi, dz = sx[2][jj] - zi;
            pot += sm[jj] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
        }
    }
    double e = 0.0;
    if (live) {
        const double vx = v[i], vy = v[ld + i], vz = v[2 * ld + i];
        e = m[i] * (0.5 * (vx * vx + vy * vy + vz * vz) - 0.5 * G * pot);
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Sum of the block partials in a fixed order (one block).
__global__ void k_sum(int64_t n, const double *partial, double *out)
{
    __shared__ double red[kDiagThreads];
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += partial[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// mu e = (|v|^2 - mu/|r|) r - (r.v) v with r, v relative to the central body.
__global__ void k_ecc(int64_t N, int64_t ld, const double *m, const double *x, const double *v,
                      double G, int central, double *e)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (i == central) {
        for (int c = 0; c < 3; ++c) e[c * ld + i] = 0.0;
        return;
    }
    double r[3], u[3];
    for (int c = 0; c < 3; ++c) {
        r[c] = x[c * ld + i] - x[c * ld + central];
        u[c] = v[c * ld + i] - v[c * ld + central];
    }
    const double mu = G * (m[central] + m[i]);
    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double v2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double rv = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
    for (int c = 0; c < 3; ++c) e[c * ld + i] = ((v2 - mu / rn) * r[c] - rv * u[c]) / mu;
}

}  // namespace

size_t energy_scratch_doubles(int64_t N) { return (size_t)((N + kDiagThreads - 1) / kDiagThreads) + 1; }

int launch_energy(const DeviceState &s, double eps, double G, double *scratch, double *e_dev,
                  cudaStream_t st)
{
    const int64_t nb = (s.N + kDiagThreads - 1) / kDiagThreads;
    k_energy<<<(unsigned)nb, kDiagThreads, 0, st>>>(s.N, s.Np, s.m, s.x0, s.v0, eps * eps, G, scratch);
    MH_LAUNCHED("k_energy");
    k_sum<<<1, kDiagThreads, 0, st>>>(nb, scratch, e_dev);
    MH_LAUNCHED("k_sum");
    return MH_OK;
}

int launch_ecc(const DeviceState &s, double G, int central, double *ecc, cudaStream_t st)
{
    k_ecc<<<(unsigned)((s.N + 127) / 128), 128, 0, st>>>(s.N, s.Np, s.m, s.x0, s.v0, G, central, ecc);
    MH_LAUNCHED("k_ecc");
    return MH_OK;
}

}  // namespace mh
