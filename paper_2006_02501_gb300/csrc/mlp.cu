// Small multilayer perceptron n_in -> H -> H -> n_out (SiLU) trained and run
// on the GPU with BF16 inputs and FP32 accumulation: the learned residual on
// the Taylor predictor.  The paper has no learned component; the network is a
// workload-side addition documented with the design.
//
// Every product is one GEMM kernel on the tensor cores, mma.sync m16n8k16 with
// bf16 operands and fp32 accumulators; operands are staged through shared
// memory in the fragment-friendly layout, which also absorbs the transposes of
// the backward pass.  Elementwise kernels apply bias and activation, form the
// mean-squared-error gradient, sum bias gradients and take the Adam step
// (Kingma & Ba 2015) on an FP32 master copy of the parameters, refreshed into
// bf16 after every step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "common.cuh"

namespace mh {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTM = 64, kTN = 64, kTK = 16, kPadK = 8;

// C[M x N] (fp32, row stride ldc) = A[M x K] B[K x N] with bf16 operands:
//   A(m, k) = TA ? a[k * lda + m] : a[m * lda + k]
//   B(k, n) = TB ? b[n * ldb + k] : b[k * ldb + n]
template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const bf16 *__restrict__ a, int lda,
                                                   const bf16 *__restrict__ b, int ldb, float *__restrict__ c,
                                                   int ldc)
{
    __shared__ __align__(16) bf16 As[kTM][kTK + kPadK];     // [m][k]
    __shared__ __align__(16) bf16 Bs[kTN][kTK + kPadK];     // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    const bf16 zero = __float2bfloat16(0.0f);
    for (int k0 = 0; k0 < K; k0 += kTK) {
        for (int e = tid; e < kTM * kTK; e += 128) {
            const int r = e / kTK, kk = e - r * kTK;
            const int k = k0 + kk;
            const int m = m0 + r, n = n0 + r;
            As[r][kk] = (m < M && k < K) ? (TA ? a[(size_t)k * lda + m] : a[(size_t)m * lda + k]) : zero;
            Bs[r][kk] = (n < N && k < K) ? (TB ? b[(size_t)n * ldb + k] : b[(size_t)k * ldb + n]) : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i;
            af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r + g][2 * t]);
            af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + g + 8][2 * t]);
            af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r + g][2 * t + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + g + 8][2 * t + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cn = wn + 8 * j;
            bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[cn + g][2 * t]);
            bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[cn + g][2 * t + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                      "r"(bfr[j][1]));
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (q & 1);
                if (m < M && n < N) c[(size_t)m * ldc + n] = acc[i][j][q];
            }
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// Z += b (per column); act: H = bf16(silu(Z)) (H may be null for the output layer).
__global__ void k_bias_act(int64_t B, int N, float *Z, const float *bias, bf16 *H, int act)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * N) return;
    const float z = Z[e] + bias[e % N];
    Z[e] = z;
    if (H) H[e] = __float2bfloat16(act ? silu(z) : z);
}

// dZ = bf16(dH * silu'(Z))
__global__ void k_dact(int64_t n, const float *dH, const float *Z, bf16 *dZ)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    dZ[e] = __float2bfloat16(dH[e] * dsilu(Z[e]));
}

// dY = bf16(2 (Y - T) / (B n_out)); per-block partial sums of (Y - T)^2 (double).
__global__ void k_mse(int64_t n, int64_t denom, const float *Y, const float *T, bf16 *dY, double *part)
{
    __shared__ double red[256];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (e < n) {
        const float d = Y[e] - T[e];
        dY[e] = __float2bfloat16(2.0f * d / (float)denom);
        s = (double)d * (double)d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_double(int64_t n, const double *x, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += x[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// out[n] = sum_b X[b][n] (bf16 inputs, fp32 sum in a fixed order per column)
__global__ void k_colsum(int64_t B, int N, const bf16 *X, float *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int64_t b = 0; b < B; ++b) s += __bfloat162float(X[b * N + n]);
    out[n] = s;
}

// rows of src (fp32, width w) gathered by idx (or 0..n-1) into bf16 / fp32 dst
__global__ void k_gather(int64_t n, int w, const float *src, const int *idx, bf16 *dst16, float *dst32)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * w) return;
    const int64_t r = e / w, c = e - r * w;
    const int64_t s = idx ? (int64_t)idx[r] : r;
    const float v = src[s * w + c];
    if (dst16) dst16[e] = __float2bfloat16(v);
    if (dst32) dst32[e] = v;
}

__global__ void k_adam(int64_t n, float *p, const float *g, float *m, float *v, bf16 *p16, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gr = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gr;
    const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float q = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = q;
    p16[e] = __float2bfloat16(q);
}

__global__ void k_to_bf16(int64_t n, const float *x, bf16 *y)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = __float2bfloat16(x[e]);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <bool TA, bool TB>
int gemm(int M, int N, int K, const bf16 *a, int lda, const bf16 *b, int ldb, float *c, int ldc, cudaStream_t st)
{
    dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
    k_gemm_bf16<TA, TB><<<grid, 128, 0, st>>>(M, N, K, a, lda, b, ldb, c, ldc);
    MH_LAUNCHED("k_gemm_bf16");
    return MH_OK;
}

}  // namespace
}  // namespace mh

using namespace mh;

struct mh_mlp {
    int n_in = 0, H = 0, n_out = 0;
    int64_t n_params = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *p16 = nullptr;
    int64_t t = 0;
    int64_t cap = 0;                 // rows of the workspace
    bf16 *X16 = nullptr, *H1 = nullptr, *H2 = nullptr, *dY16 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *T = nullptr, *dH2 = nullptr, *dH1 = nullptr;
    double *lpart = nullptr, *lsum = nullptr;
    int *idx = nullptr;
    int64_t idx_cap = 0;
};

namespace {

void free_ws(mh_mlp *n)
{
    void *ptrs[] = {n->X16, n->H1, n->H2, n->dY16, n->dZ2, n->dZ1, n->Z1, n->Z2, n->Y, n->T, n->dH2, n->dH1, n->lpart, n->lsum};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    n->X16 = n->H1 = n->H2 = n->dY16 = n->dZ2 = n->dZ1 = nullptr;
    n->Z1 = n->Z2 = n->Y = n->T = n->dH2 = n->dH1 = nullptr;
    n->lpart = n->lsum = nullptr;
    n->cap = 0;
}

int ensure_ws(mh_mlp *n, int64_t rows, cudaStream_t st)
{
    if (rows <= n->cap) return MH_OK;
    MH_CUDA(cudaStreamSynchronize(st));
    free_ws(n);
    const int64_t H = n->H;
    MH_CUDA(cudaMalloc((void **)&n->X16, rows * n->n_in * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->H1, rows * H * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->H2, rows * H * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->dY16, rows * n->n_out * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->dZ2, rows * H * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->dZ1, rows * H * sizeof(bf16)));
    MH_CUDA(cudaMalloc((void **)&n->Z1, rows * H * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->Z2, rows * H * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->Y, rows * n->n_out * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->T, rows * n->n_out * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->dH2, rows * H * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->dH1, rows * H * sizeof(float)));
    MH_CUDA(cudaMalloc((void **)&n->lpart, (nb(rows * n->n_out) + 1) * sizeof(double)));
    MH_CUDA(cudaMalloc((void **)&n->lsum, sizeof(double)));
    n->cap = rows;
    return MH_OK;
}

// Forward over rows already gathered into X16; Y (fp32) holds the outputs.
int forward_ws(mh_mlp *n, int64_t B, cudaStream_t st)
{
    const int H = n->H;
    const bf16 *W1 = n->p16 + n->oW1, *W2 = n->p16 + n->oW2, *W3 = n->p16 + n->oW3;
    if (int rc = gemm<false, true>((int)B, H, n->n_in, n->X16, n->n_in, W1, n->n_in, n->Z1, H, st)) return rc;
    k_bias_act<<<nb(B * H), 256, 0, st>>>(B, H, n->Z1, n->p + n->ob1, n->H1, 1);
    MH_LAUNCHED("k_bias_act");
    if (int rc = gemm<false, true>((int)B, H, H, n->H1, H, W2, H, n->Z2, H, st)) return rc;
    k_bias_act<<<nb(B * H), 256, 0, st>>>(B, H, n->Z2, n->p + n->ob2, n->H2, 1);
    MH_LAUNCHED("k_bias_act");
    if (int rc = gemm<false, true>((int)B, n->n_out, H, n->H2, H, W3, H, n->Y, n->n_out, st)) return rc;
    k_bias_act<<<nb(B * n->n_out), 256, 0, st>>>(B, n->n_out, n->Y, n->p + n->ob3, nullptr, 0);
    MH_LAUNCHED("k_bias_act");
    return MH_OK;
}

// Loss (device scalar lsum, sum of squares) and gradients into g, for rows in X16 / T.
int backward_ws(mh_mlp *n, int64_t B, cudaStream_t st)
{
    const int H = n->H, O = n->n_out;
    const bf16 *W2 = n->p16 + n->oW2, *W3 = n->p16 + n->oW3;
    const int64_t ny = B * O;
    k_mse<<<nb(ny), 256, 0, st>>>(ny, ny, n->Y, n->T, n->dY16, n->lpart);
    MH_LAUNCHED("k_mse");
    k_sum_double<<<1, 256, 0, st>>>(nb(ny), n->lpart, n->lsum);
    MH_LAUNCHED("k_sum_double");
    // output layer
    if (int rc = gemm<true, false>(O, H, (int)B, n->dY16, O, n->H2, H, n->g + n->oW3, H, st)) return rc;
    k_colsum<<<nb(O, 128), 128, 0, st>>>(B, O, n->dY16, n->g + n->ob3);
    MH_LAUNCHED("k_colsum");
    if (int rc = gemm<false, false>((int)B, H, O, n->dY16, O, W3, H, n->dH2, H, st)) return rc;
    k_dact<<<nb(B * H), 256, 0, st>>>(B * H, n->dH2, n->Z2, n->dZ2);
    MH_LAUNCHED("k_dact");
    // hidden layer 2
    if (int rc = gemm<true, false>(H, H, (int)B, n->dZ2, H, n->H1, H, n->g + n->oW2, H, st)) return rc;
    k_colsum<<<nb(H, 128), 128, 0, st>>>(B, H, n->dZ2, n->g + n->ob2);
    MH_LAUNCHED("k_colsum");
    if (int rc = gemm<false, false>((int)B, H, H, n->dZ2, H, W2, H, n->dH1, H, st)) return rc;
    k_dact<<<nb(B * H), 256, 0, st>>>(B * H, n->dH1, n->Z1, n->dZ1);
    MH_LAUNCHED("k_dact");
    // hidden layer 1
    if (int rc = gemm<true, false>(H, n->n_in, (int)B, n->dZ1, H, n->X16, n->n_in, n->g + n->oW1, n->n_in, st)) return rc;
    k_colsum<<<nb(H, 128), 128, 0, st>>>(B, H, n->dZ1, n->g + n->ob1);
    MH_LAUNCHED("k_colsum");
    return MH_OK;
}

int check_net(const mh_mlp *n)
{
    if (!n) { set_error("NULL mh_mlp handle"); return MH_EINVAL; }
    return MH_OK;
}

}  // namespace

namespace mh {
// Inference for the learned predictor (learned.cu): Y[n x n_out] from X[n x n_in] (fp32, device).
int mlp_infer(mh_mlp *n, const float *X, float *Y, int64_t rows, cudaStream_t st)
{
    const int64_t chunk = 65536;
    if (int rc = ensure_ws(n, std::min(rows, chunk), st)) return rc;
    for (int64_t r0 = 0; r0 < rows; r0 += chunk) {
        const int64_t B = std::min(chunk, rows - r0);
        k_gather<<<nb(B * n->n_in), 256, 0, st>>>(B, n->n_in, X + r0 * n->n_in, nullptr, n->X16, nullptr);
        MH_LAUNCHED("k_gather");
        if (int rc = forward_ws(n, B, st)) return rc;
        MH_CUDA(cudaMemcpyAsync(Y + r0 * n->n_out, n->Y, B * n->n_out * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return MH_OK;
}
int mlp_dims(const mh_mlp *n, int *n_in, int *n_out)
{
    if (!n) return MH_EINVAL;
    *n_in = n->n_in;
    *n_out = n->n_out;
    return MH_OK;
}
}  // namespace mh

extern "C" {

int mh_mlp_create(mh_mlp **out, int n_in, int n_hidden, int n_out, uint64_t seed)
{
    if (!out) { set_error("mh_mlp_create: out is NULL"); return MH_EINVAL; }
    *out = nullptr;
    if (n_in < 1 || n_in > 4096 || n_hidden < 1 || n_hidden > 4096 || n_out < 1 || n_out > 4096) {
        set_error("mh_mlp_create: sizes must be in [1, 4096]");
        return MH_EINVAL;
    }
    mh_mlp *n = new (std::nothrow) mh_mlp();
    if (!n) { set_error("mh_mlp_create: host allocation failed"); return MH_ENOMEM; }
    n->n_in = n_in;
    n->H = n_hidden;
    n->n_out = n_out;
    n->oW1 = 0;
    n->ob1 = n->oW1 + (int64_t)n_hidden * n_in;
    n->oW2 = n->ob1 + n_hidden;
    n->ob2 = n->oW2 + (int64_t)n_hidden * n_hidden;
    n->oW3 = n->ob2 + n_hidden;
    n->ob3 = n->oW3 + (int64_t)n_out * n_hidden;
    n->n_params = n->ob3 + n_out;
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    std::vector<float> h(n->n_params, 0.0f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<float> u(-1.0f, 1.0f);
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        const float sc = 1.0f / std::sqrt((float)fan_in);
        for (int64_t k = 0; k < count; ++k) h[off + k] = sc * u(rng);
    };
    fill(n->oW1, (int64_t)n_hidden * n_in, n_in);
    fill(n->oW2, (int64_t)n_hidden * n_hidden, n_hidden);
    fill(n->oW3, (int64_t)n_out * n_hidden, n_hidden);
    cudaError_t e = cudaMalloc((void **)&n->p, n->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->g, n->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->m, n->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->v, n->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->p16, n->n_params * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMemcpy(n->p, h.data(), n->n_params * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->n_params * sizeof(float));
    if (e == cudaSuccess) {
        k_to_bf16<<<nb(n->n_params), 256>>>(n->n_params, n->p, n->p16);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "mh_mlp_create");
        mh_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return MH_OK;
}

void mh_mlp_destroy(mh_mlp *n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    free_ws(n);
    void *ptrs[] = {n->p, n->g, n->m, n->v, n->p16, n->idx};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete n;
}

int mh_mlp_num_params(const mh_mlp *n, int64_t *count)
{
    if (int rc = check_net(n)) return rc;
    if (count) *count = n->n_params;
    return MH_OK;
}

int mh_mlp_get_params(mh_mlp *n, float *host, int64_t count)
{
    if (int rc = check_net(n)) return rc;
    if (!host || count != n->n_params) { set_error("mh_mlp_get_params: need n_params floats"); return MH_EINVAL; }
    MH_CUDA(cudaDeviceSynchronize());
    MH_CUDA(cudaMemcpy(host, n->p, count * sizeof(float), cudaMemcpyDeviceToHost));
    return MH_OK;
}

int mh_mlp_set_params(mh_mlp *n, const float *host, int64_t count)
{
    if (int rc = check_net(n)) return rc;
    if (!host || count != n->n_params) { set_error("mh_mlp_set_params: need n_params floats"); return MH_EINVAL; }
    MH_CUDA(cudaDeviceSynchronize());
    MH_CUDA(cudaMemcpy(n->p, host, count * sizeof(float), cudaMemcpyHostToDevice));
    MH_CUDA(cudaMemset(n->m, 0, count * sizeof(float)));
    MH_CUDA(cudaMemset(n->v, 0, count * sizeof(float)));
    n->t = 0;
    k_to_bf16<<<nb(count), 256>>>(count, n->p, n->p16);
    MH_LAUNCHED("k_to_bf16");
    MH_CUDA(cudaDeviceSynchronize());
    return MH_OK;
}

int mh_mlp_forward(mh_mlp *n, const float *x, float *y, int64_t rows, void *stream)
{
    if (int rc = check_net(n)) return rc;
    if (!x || !y || rows < 1) { set_error("mh_mlp_forward: device x, y and rows >= 1 required"); return MH_EINVAL; }
    return mlp_infer(n, x, y, rows, (cudaStream_t)stream);
}

int mh_mlp_loss_grad(mh_mlp *n, const float *x, const float *t, int64_t rows, double *loss, float *grad_host,
                     void *stream)
{
    if (int rc = check_net(n)) return rc;
    if (!x || !t || rows < 1 || rows > (1 << 24)) { set_error("mh_mlp_loss_grad: device x, t and 1 <= rows <= 2^24"); return MH_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = ensure_ws(n, rows, st)) return rc;
    k_gather<<<nb(rows * n->n_in), 256, 0, st>>>(rows, n->n_in, x, nullptr, n->X16, nullptr);
    MH_LAUNCHED("k_gather");
    k_gather<<<nb(rows * n->n_out), 256, 0, st>>>(rows, n->n_out, t, nullptr, nullptr, n->T);
    MH_LAUNCHED("k_gather");
    if (int rc = forward_ws(n, rows, st)) return rc;
    if (int rc = backward_ws(n, rows, st)) return rc;
    double ls = 0.0;
    MH_CUDA(cudaMemcpyAsync(&ls, n->lsum, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_host) MH_CUDA(cudaMemcpyAsync(grad_host, n->g, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, st));
    MH_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = ls / (double)(rows * n->n_out);
    return MH_OK;
}

int mh_mlp_train(mh_mlp *n, const float *x, const float *t, int64_t rows, int epochs, int batch, float lr,
                 uint64_t seed, double *final_loss, void *stream)
{
    if (int rc = check_net(n)) return rc;
    if (!x || !t || rows < 1 || epochs < 1 || batch < 1 || batch > (1 << 20) || !(lr > 0.0f)) {
        set_error("mh_mlp_train: device x, t; rows, epochs, batch >= 1; lr > 0");
        return MH_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t B = std::min<int64_t>(batch, rows);
    if (int rc = ensure_ws(n, B, st)) return rc;
    if (rows > n->idx_cap) {
        MH_CUDA(cudaStreamSynchronize(st));
        if (n->idx) cudaFree(n->idx);
        n->idx = nullptr;
        MH_CUDA(cudaMalloc((void **)&n->idx, rows * sizeof(int)));
        n->idx_cap = rows;
    }
    std::vector<int> perm(rows);
    std::iota(perm.begin(), perm.end(), 0);
    std::mt19937_64 rng(seed);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        MH_CUDA(cudaMemcpyAsync(n->idx, perm.data(), rows * sizeof(int), cudaMemcpyHostToDevice, st));
        double ep_sum = 0.0;
        int64_t ep_rows = 0;
        for (int64_t r0 = 0; r0 + B <= rows; r0 += B) {      // the ragged tail is left to the next epoch's order
            k_gather<<<nb(B * n->n_in), 256, 0, st>>>(B, n->n_in, x, n->idx + r0, n->X16, nullptr);
            MH_LAUNCHED("k_gather");
            k_gather<<<nb(B * n->n_out), 256, 0, st>>>(B, n->n_out, t, n->idx + r0, nullptr, n->T);
            MH_LAUNCHED("k_gather");
            if (int rc = forward_ws(n, B, st)) return rc;
            if (int rc = backward_ws(n, B, st)) return rc;
            n->t += 1;
            const float c1 = 1.0f - std::pow(0.9f, (float)n->t), c2 = 1.0f - std::pow(0.999f, (float)n->t);
            k_adam<<<nb(n->n_params), 256, 0, st>>>(n->n_params, n->p, n->g, n->m, n->v, n->p16, lr, 0.9f, 0.999f,
                                                    1e-8f, c1, c2);
            MH_LAUNCHED("k_adam");
            double ls = 0.0;
            if (r0 + 2 * B > rows) {           // last batch of the epoch: read its loss
                MH_CUDA(cudaMemcpyAsync(&ls, n->lsum, sizeof(double), cudaMemcpyDeviceToHost, st));
                MH_CUDA(cudaStreamSynchronize(st));
                ep_sum += ls;
                ep_rows += B;
            }
        }
        if (ep_rows) last = ep_sum / (double)(ep_rows * n->n_out);
    }
    MH_CUDA(cudaStreamSynchronize(st));
    if (final_loss) *final_loss = last;
    return MH_OK;
}

}  // extern "C"
