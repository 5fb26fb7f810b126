// Batched integrator: thousands of independent small systems (up to 64 bodies
// each) advanced by the shared-step P(EC)^n scheme in one persistent launch.
//
// Mapping: one warp integrates one system at a time, for all requested steps,
// without any synchronisation beyond the warp.  Lane l owns bodies l and l+32
// (x, v and a^(0..2p-1) in registers); the evaluation spreads each body's
// sources over a group of lanes where the system leaves lanes idle
// (eval_group); the evaluation inputs of the whole
// system (x, v, a, a-dot and G m of every body) sit in two shared-memory
// buffers that alternate between the passes of P(EC)^n, so a lane can write
// its corrected bodies while others still read the previous ones.  Warps take
// systems from a work queue (one atomic per system) in an order chosen by the
// autotuner (largest systems first, or as given), which balances the O(N_s^2)
// work across the 152 SMs.  Results do not depend on which warp runs a system.
//
// The step is the same as the single-system path: Taylor predictor, n_iter
// evaluations with the corrector of Eqs. 6-7 (beta of Eq. 20 or 1), then the
// Hermite interpolation of a^(p+1..2p-1); the evaluation of body i sums the
// pair derivatives over all j != i of its own system (FP64).
#include <algorithm>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "hermite_step.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

constexpr int kBatchMax = 64;     // bodies per system (two per lane)

struct BatchArgs {
    int S;
    const int64_t *off;       // [S+1] body offsets of the systems
    const int *order;         // [S] work order
    const double *dt;         // [S] step of each system
    const double *m;          // [ld]
    double *x, *v, *d;        // [3][ld], [3][ld], [2p][3][ld]
    int64_t ld;
    double eps2, G;
    int n_steps, n_iter, beta_mode, init;
    int *counter;             // work queue head
    int *flag;                // non-finite flag
};

template <int p>
__host__ __device__ constexpr int rows_init() { return 6 * p; }        // x, v, a .. a^(2p-3): 3(P+1) rows for P = 2p-1
template <int p>
__host__ __device__ constexpr int rows_step() { return 3 * (p + 1); }  // x, v, a, a-dot as the evaluation needs

// Shared-memory doubles per warp: G m row, the initialisation/first buffer, the second buffer.
template <int p>
__host__ __device__ constexpr int smem_per_warp() { return kBatchMax * (1 + rows_init<p>() + rows_step<p>()); }

// a^(0..P) of body i of a system of n bodies from input rows `in` (stride kBatchMax).
template <int P>
__device__ __forceinline__ void eval_body(const double *in, const double *gm, int n, int i, double eps2,
                                          double (&acc)[P + 1][3])
{
    double ri[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ri[k][c] = in[(3 * k + c) * kBatchMax + i];
            acc[k][c] = 0.0;
        }
    for (int j = 0; j < n; ++j) {
        double r[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = in[(3 * k + c) * kBatchMax + j] - ri[k][c];
        const bool self = j == i;
        double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], eps2)));
        s = self ? 1.0 : s;
        const double mj = self ? 0.0 : gm[j];
        const double rinv = rsqrt_fp64(s);
        const double sinv = rinv * rinv;
        pair_derivs<P, double>(r, mj * (rinv * sinv), sinv, acc);
    }
}

// a^(0..P) of bodies base .. base + m - 1 (m <= 32) of a system of n bodies by
// the whole warp: each body gets a group of g lanes (g the largest power of two
// with g m <= 32), lane l works on body base + l / g over the sources j = l % g,
// l % g + g, ..., the group's sums meet in a fixed xor tree, and lane l returns
// the sums of body base + l (its own body; lanes l >= m get garbage).  Every
// body's sum is taken in an order fixed by n alone, so results do not depend on
// the warp.  Systems that leave lanes idle (n < 32, or the second half of one of
// 33 .. 64 bodies) spread their pairs over the idle lanes.
template <int P>
__device__ __forceinline__ void eval_group(const double *in, const double *gm, int n, int base, int m, int lane,
                                           double eps2, double (&out)[P + 1][3])
{
    int g = 1;
    while (2 * g * m <= 32) g *= 2;
    const int k0 = lane / g, sub = lane % g;
    const int i = base + (k0 < m ? k0 : 0);
    double ri[P + 1][3], acc[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ri[k][c] = in[(3 * k + c) * kBatchMax + i];
            acc[k][c] = 0.0;
        }
    for (int j = sub; j < n; j += g) {
        double r[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = in[(3 * k + c) * kBatchMax + j] - ri[k][c];
        const bool self = j == i;
        double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], eps2)));
        s = self ? 1.0 : s;
        const double mj = self ? 0.0 : gm[j];
        const double rinv = rsqrt_fp64(s);
        const double sinv = rinv * rinv;
        pair_derivs<P, double>(r, mj * (rinv * sinv), sinv, acc);
    }
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = acc[k][c];
            for (int o = 1; o < g; o *= 2) v += __shfl_xor_sync(0xffffffffu, v, o);
            out[k][c] = __shfl_sync(0xffffffffu, v, (lane * g) & 31);
        }
}

// One initialisation pass: a^(have .. min(have+1, 2p-1)) from x, v, a^(0..have-1).
template <int p, int have>
__device__ __forceinline__ void init_pass(double *in, const double *gm, int n, int lane, double eps2,
                                          double (&x0)[2][3], double (&v0)[2][3], double (&d0)[2][2 * p][3])
{
    constexpr int P = have + 1;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int i = lane + 32 * b;
        if (i < n)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                in[c * kBatchMax + i] = x0[b][c];
                in[(3 + c) * kBatchMax + i] = v0[b][c];
#pragma unroll
                for (int k = 0; k < have; ++k) in[(6 + 3 * k + c) * kBatchMax + i] = d0[b][k][c];
            }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int i = lane + 32 * b;
        if (i < n) {
            double acc[P + 1][3];
            eval_body<P>(in, gm, n, i, eps2, acc);
#pragma unroll
            for (int k = have; k <= P && k < 2 * p; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) d0[b][k][c] = acc[k][c];
        }
    }
    __syncwarp();
}

template <int p>
__global__ void __launch_bounds__(256) k_batch(BatchArgs a)
{
    constexpr int K = 2 * p;
    constexpr int RS = rows_step<p>();
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *gm = smem + (size_t)warp * smem_per_warp<p>();
    double *bufA = gm + kBatchMax;
    double *bufB = bufA + kBatchMax * rows_init<p>();

    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.counter, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= a.S) break;
        const int sys = a.order[idx];
        const int64_t o = a.off[sys];
        const int n = (int)(a.off[sys + 1] - o);
        const double dt = a.dt[sys];

        double x0[2][3], v0[2][3], d0[2][K][3];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = lane + 32 * b;
            const int64_t g = o + (i < n ? i : 0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x0[b][c] = a.x[c * a.ld + g];
                v0[b][c] = a.v[c * a.ld + g];
#pragma unroll
                for (int k = 0; k < K; ++k) d0[b][k][c] = a.init ? 0.0 : a.d[(3 * k + c) * a.ld + g];
            }
            if (i < n) gm[i] = a.G * a.m[o + i];
        }
        __syncwarp();
        if (a.init) {
            init_pass<p, 0>(bufA, gm, n, lane, a.eps2, x0, v0, d0);
            if constexpr (p >= 2) init_pass<p, 2>(bufA, gm, n, lane, a.eps2, x0, v0, d0);
            if constexpr (p >= 3) init_pass<p, 4>(bufA, gm, n, lane, a.eps2, x0, v0, d0);
        }

        bool finite = true;
        for (int step = 0; step < a.n_steps; ++step) {
            double *cur = bufA, *nxt = bufB;
            // predictor: every body's evaluation input at t0 + dt
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int i = lane + 32 * b;
                if (i < n)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        double dk[K], xp, vp, ad[p > 1 ? p - 1 : 1];
#pragma unroll
                        for (int k = 0; k < K; ++k) dk[k] = d0[b][k][c];
                        predict_comp<p>(dt, dk, x0[b][c], v0[b][c], xp, vp, ad);
                        cur[c * kBatchMax + i] = xp;
                        cur[(3 + c) * kBatchMax + i] = vp;
#pragma unroll
                        for (int q = 0; q + 2 <= p; ++q) cur[(6 + 3 * q + c) * kBatchMax + i] = ad[q];
                    }
            }
            __syncwarp();
            for (int it = 0; it < a.n_iter; ++it) {
                const bool last = it == a.n_iter - 1;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int i = lane + 32 * b;
                    if (32 * b >= n) continue;           // the whole warp: n is the system's
                    double acc[p + 1][3];
                    eval_group<p>(cur, gm, n, 32 * b, min(n - 32 * b, 32), lane, a.eps2, acc);
                    if (i >= n) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        double dk[K], d1[p + 1], xn, vn;
#pragma unroll
                        for (int k = 0; k < K; ++k) dk[k] = d0[b][k][c];
#pragma unroll
                        for (int k = 0; k <= p; ++k) d1[k] = acc[k][c];
                        correct_comp<p>(dt, a.beta_mode, dk, d1, x0[b][c], v0[b][c], xn, vn);
                        finite = finite && isfinite(xn) && isfinite(vn);
                        if (!last) {
                            nxt[c * kBatchMax + i] = xn;
                            nxt[(3 + c) * kBatchMax + i] = vn;
#pragma unroll
                            for (int q = 0; q + 2 <= p; ++q) nxt[(6 + 3 * q + c) * kBatchMax + i] = d1[q];
                        } else {
                            double hi[K > p + 1 ? p - 1 : 1];
                            interp_comp<p>(dt, dk, d1, hi);
                            x0[b][c] = xn;
                            v0[b][c] = vn;
#pragma unroll
                            for (int k = 0; k < K; ++k) d0[b][k][c] = k <= p ? d1[k] : hi[k - p - 1];
                        }
                    }
                }
                __syncwarp();
                double *t = cur;
                cur = nxt;
                nxt = t;
            }
        }
        if (!finite) atomicOr(a.flag, 1);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = lane + 32 * b;
            if (i < n) {
                const int64_t g = o + i;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a.x[c * a.ld + g] = x0[b][c];
                    a.v[c * a.ld + g] = v0[b][c];
#pragma unroll
                    for (int k = 0; k < K; ++k) a.d[(3 * k + c) * a.ld + g] = d0[b][k][c];
                }
            }
        }
        __syncwarp();
    }
}

// Energy of each system (one warp per system): sum m v^2/2 - sum_{i<j} G m_i m_j / sqrt(r^2 + eps^2).
__global__ void k_batch_energy(int S, const int64_t *off, const double *m, const double *x, const double *v,
                               int64_t ld, double eps2, double G, double *E)
{
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= S) return;
    const int64_t o = off[warp];
    const int n = (int)(off[warp + 1] - o);
    double e = 0.0;
    for (int i = lane; i < n; i += 32) {
        const int64_t gi = o + i;
        const double vx = v[gi], vy = v[ld + gi], vz = v[2 * ld + gi];
        double pot = 0.0;
        for (int j = i + 1; j < n; ++j) {
            const int64_t gj = o + j;
            const double dx = x[gj] - x[gi], dy = x[ld + gj] - x[ld + gi], dz = x[2 * ld + gj] - x[2 * ld + gi];
            pot += m[gj] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
        }
        e += m[gi] * (0.5 * (vx * vx + vy * vy + vz * vz) - G * pot);
    }
    for (int s = 16; s > 0; s >>= 1) e += __shfl_xor_sync(0xffffffffu, e, s);
    if (lane == 0) E[warp] = e;
}

template <int p>
int launch_batch_p(const BatchArgs &a, int warps, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)smem_per_warp<p>() * warps;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        MH_CUDA(cudaFuncSetAttribute(k_batch<p>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set[dev] = true;
    }
    int n_sm = 0;
    MH_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    MH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<p>, 32 * warps, smem));
    if (per_sm < 1) {
        set_error("batched integrator: launch configuration does not fit an SM");
        return MH_EINVAL;
    }
    const int grid = std::min(n_sm * per_sm, (a.S + warps - 1) / warps);
    k_batch<p><<<std::max(grid, 1), 32 * warps, smem, st>>>(a);
    MH_LAUNCHED("k_batch");
    return MH_OK;
}

size_t batch_smem_bytes(int p, int warps)
{
    const int per = p == 1 ? smem_per_warp<1>() : p == 2 ? smem_per_warp<2>() : smem_per_warp<3>();
    return sizeof(double) * (size_t)per * warps;
}

}  // namespace

// Batch bookkeeping kept with the simulation handle.
struct BatchState {
    int S = 0;
    int64_t *off = nullptr;
    int *order = nullptr;
    double *dt = nullptr;
    int *counter = nullptr;
    double *energy = nullptr;
    std::vector<int> order_desc, order_given;
    int warps = 8;
    int order_kind = 0;         // 0 largest systems first, 1 as given
    bool tuned = false;
    std::map<std::tuple<int64_t, int, int, int>, cudaGraphExec_t> graphs;
};

}  // namespace mh

using namespace mh;

namespace {

int batch_launch(mh_sim *sim, BatchState &b, int n_steps, int n_iter, int init, double *x, double *v,
                 double *d, int warps, cudaStream_t st)
{
    DeviceState &s = sim->s;
    BatchArgs a{b.S, b.off, b.order, b.dt, s.m, x, v, d, s.Np, sim->eps * sim->eps, sim->cfg.G,
                n_steps, n_iter, sim->cfg.beta_mode, init, b.counter, s.flag};
    MH_CUDA(cudaMemsetAsync(b.counter, 0, sizeof(int), st));
    switch (s.p) {
    case 1: return launch_batch_p<1>(a, warps, st);
    case 2: return launch_batch_p<2>(a, warps, st);
    case 3: return launch_batch_p<3>(a, warps, st);
    }
    set_error("batched integrator: order must be 4, 6 or 8");
    return MH_EINVAL;
}

int set_order(BatchState &b, int kind, cudaStream_t st)
{
    const std::vector<int> &o = kind == 0 ? b.order_desc : b.order_given;
    MH_CUDA(cudaMemcpyAsync(b.order, o.data(), o.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    MH_CUDA(cudaStreamSynchronize(st));
    b.order_kind = kind;
    return MH_OK;
}

// Autotuner: time every (warps per CTA, work order) candidate on a scratch copy
// of the state for probe_steps steps and keep the fastest.  Cached per
// (order, number of systems, size histogram, device).
std::map<std::tuple<int, int, uint64_t, int>, std::pair<int, int>> g_tune_cache;

int batch_tune(mh_sim *sim, BatchState &b, int probe_steps, int n_iter)
{
    DeviceState &s = sim->s;
    std::vector<int64_t> hoff(b.S + 1);
    MH_CUDA(cudaMemcpy(hoff.data(), b.off, (b.S + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    uint64_t hist = 1469598103934665603ull;     // FNV-1a over the system sizes
    for (int k = 0; k < b.S; ++k) {
        hist ^= (uint64_t)(hoff[k + 1] - hoff[k]);
        hist *= 1099511628211ull;
    }
    const auto key = std::make_tuple(s.p, b.S, hist, sim->device);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        b.warps = it->second.first;
        b.tuned = true;
        return set_order(b, it->second.second, sim->stream);
    }
    const int K = 2 * s.p;
    double *sx = nullptr, *sv = nullptr, *sd = nullptr;
    MH_CUDA(cudaMalloc((void **)&sx, 3 * s.Np * sizeof(double)));
    MH_CUDA(cudaMalloc((void **)&sv, 3 * s.Np * sizeof(double)));
    MH_CUDA(cudaMalloc((void **)&sd, (size_t)K * 3 * s.Np * sizeof(double)));
    cudaEvent_t e0, e1;
    MH_CUDA(cudaEventCreate(&e0));
    MH_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_w = b.warps, best_o = 0;
    for (int kind = 0; kind < 2; ++kind) {
        if (int rc = set_order(b, kind, sim->stream)) return rc;
        for (int w : {2, 4, 6, 8}) {
            if (batch_smem_bytes(s.p, w) > 227 * 1024) continue;
            MH_CUDA(cudaMemcpyAsync(sx, s.x0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream));
            MH_CUDA(cudaMemcpyAsync(sv, s.v0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream));
            MH_CUDA(cudaMemcpyAsync(sd, s.d0, (size_t)K * 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice,
                                    sim->stream));
            MH_CUDA(cudaEventRecord(e0, sim->stream));
            if (int rc = batch_launch(sim, b, probe_steps, n_iter, 0, sx, sv, sd, w, sim->stream)) return rc;
            MH_CUDA(cudaEventRecord(e1, sim->stream));
            MH_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            MH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_w = w;
                best_o = kind;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sx);
    cudaFree(sv);
    cudaFree(sd);
    MH_CUDA(cudaMemsetAsync(s.flag, 0, sizeof(int), sim->stream));   // probes may not set the flag
    b.warps = best_w;
    b.tuned = true;
    g_tune_cache[key] = {best_w, best_o};
    return set_order(b, best_o, sim->stream);
}

}  // namespace

namespace mh {
void free_batch(mh_sim *sim);
}

void mh::free_batch(mh_sim *sim)
{
    BatchState *b = static_cast<BatchState *>(sim->batch);
    if (!b) return;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    void *ptrs[] = {b->off, b->order, b->dt, b->counter, b->energy};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete b;
    sim->batch = nullptr;
}

extern "C" {

int mh_create_batch(mh_sim **out, int64_t S, const int64_t *offsets, const double *m, const double *x,
                    const double *v, const double *dt, double eps, int order, const mh_config *cfg,
                    void *stream)
{
    if (!out) { set_error("mh_create_batch: out is NULL"); return MH_EINVAL; }
    *out = nullptr;
    set_error("");
    mh_config c;
    if (cfg) c = *cfg; else mh_config_default(&c);
    c.order = order;
    const int p = order == 4 ? 1 : order == 6 ? 2 : order == 8 ? 3 : 0;
    if (p == 0) { set_error("mh_create_batch: order must be 4, 6 or 8"); return MH_EINVAL; }
    if (S < 1 || S > (1 << 30) || !offsets || !m || !x || !v || !dt) {
        set_error("mh_create_batch: need S >= 1 and non-NULL offsets, m, x, v, dt");
        return MH_EINVAL;
    }
    if (offsets[0] != 0) { set_error("mh_create_batch: offsets[0] must be 0"); return MH_EINVAL; }
    for (int64_t k = 0; k < S; ++k) {
        const int64_t n = offsets[k + 1] - offsets[k];
        if (n < 1 || n > kBatchMax) {
            set_error("mh_create_batch: every system needs 1 to 64 bodies");
            return MH_EINVAL;
        }
        if (!(dt[k] != 0.0) || !std::isfinite(dt[k])) { set_error("mh_create_batch: dt must be finite and non-zero"); return MH_EINVAL; }
    }
    if (c.precision != MH_PREC_FP64) { set_error("mh_create_batch: the batched integrator runs in FP64"); return MH_EINVAL; }
    if (c.step_mode != MH_STEP_SHARED) { set_error("mh_create_batch: shared steps only"); return MH_EINVAL; }
    const int64_t N = offsets[S];
    // the per-body arrays, the device stream and the state layout of a single system
    mh_config c1 = c;
    int rc = mh_create_shell(out, N, order, m, x, v, eps, &c1, stream);
    if (rc) return rc;
    mh_sim *sim = *out;
    BatchState *b = new (std::nothrow) BatchState();
    if (!b) { mh_destroy(sim); *out = nullptr; set_error("mh_create_batch: host allocation failed"); return MH_ENOMEM; }
    sim->batch = b;
    b->S = (int)S;
    b->order_given.resize(S);
    std::iota(b->order_given.begin(), b->order_given.end(), 0);
    b->order_desc = b->order_given;
    std::stable_sort(b->order_desc.begin(), b->order_desc.end(), [&](int i, int j) {
        return offsets[i + 1] - offsets[i] > offsets[j + 1] - offsets[j];
    });
    auto fail = [&](int r) { mh_destroy(sim); *out = nullptr; return r; };
    cudaError_t e = cudaMalloc((void **)&b->off, (S + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->order, S * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->dt, S * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->energy, S * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->off, offsets, (S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, sim->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dt, dt, S * sizeof(double), cudaMemcpyHostToDevice, sim->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "mh_create_batch: allocation"));
    if ((rc = set_order(*b, 0, sim->stream))) return fail(rc);
    // a^(0..2p-1) of every body at t = 0, per system (Section 3 intro)
    if ((rc = batch_launch(sim, *b, 0, 1, 1, sim->s.x0, sim->s.v0, sim->s.d0, b->warps, sim->stream))) return fail(rc);
    e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "mh_create_batch: initialisation"));
    return MH_OK;
}

int mh_batch_tune(mh_sim *sim, int probe_steps, int n_iter, int *warps, int *order_kind)
{
    if (!sim || !sim->batch) { set_error("mh_batch_tune: not a batched simulation"); return MH_EINVAL; }
    if (probe_steps < 1 || n_iter < 1 || n_iter > 64) { set_error("mh_batch_tune: probe_steps >= 1, 1 <= n_iter <= 64"); return MH_EINVAL; }
    BatchState &b = *static_cast<BatchState *>(sim->batch);
    if (int rc = batch_tune(sim, b, probe_steps, n_iter)) return rc;
    if (warps) *warps = b.warps;
    if (order_kind) *order_kind = b.order_kind;
    return MH_OK;
}

int mh_step_batch(mh_sim *sim, int64_t n_steps, int n_iter)
{
    if (!sim || !sim->batch) { set_error("mh_step_batch: not a batched simulation"); return MH_EINVAL; }
    if (n_steps < 1 || n_steps > (1 << 30) || n_iter < 1 || n_iter > 64) {
        set_error("mh_step_batch: need 1 <= n_steps <= 2^30 and 1 <= n_iter <= 64");
        return MH_EINVAL;
    }
    NvtxScope range("mh_step_batch");
    BatchState &b = *static_cast<BatchState *>(sim->batch);
    if (!b.tuned)
        if (int rc = batch_tune(sim, b, (int)std::min<int64_t>(n_steps, 8), n_iter)) return rc;
    // one persistent launch, captured once per (steps, passes, configuration) as a CUDA graph
    const auto key = std::make_tuple(n_steps, n_iter, b.warps, b.order_kind);
    auto it = b.graphs.find(key);
    if (it == b.graphs.end()) {
        cudaGraph_t g = nullptr;
        MH_CUDA(cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal));
        int rc = batch_launch(sim, b, (int)n_steps, n_iter, 0, sim->s.x0, sim->s.v0, sim->s.d0, b.warps, sim->stream);
        cudaError_t e = cudaStreamEndCapture(sim->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "mh_step_batch: stream capture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "mh_step_batch: graph instantiation");
        it = b.graphs.emplace(key, ex).first;
    }
    MH_CUDA(cudaGraphLaunch(it->second, sim->stream));
    sim->ctr.steps += n_steps;
    sim->ctr.kernel_launches += 1;
    sim->ctr.evaluations += n_steps * n_iter;
    sim->ctr.particle_steps += (double)n_steps * (double)sim->s.N;
    return MH_OK;
}

int mh_batch_energy(mh_sim *sim, double *energy)
{
    if (!sim || !sim->batch || !energy) { set_error("mh_batch_energy: batched simulation and output required"); return MH_EINVAL; }
    BatchState &b = *static_cast<BatchState *>(sim->batch);
    DeviceState &s = sim->s;
    const int threads = 256;
    const unsigned blocks = (unsigned)(((int64_t)b.S * 32 + threads - 1) / threads);
    k_batch_energy<<<blocks, threads, 0, sim->stream>>>(b.S, b.off, s.m, s.x0, s.v0, s.Np, sim->eps * sim->eps,
                                                        sim->cfg.G, b.energy);
    MH_LAUNCHED("k_batch_energy");
    MH_CUDA(cudaMemcpyAsync(energy, b.energy, b.S * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    sim->ctr.kernel_launches += 1;
    return MH_OK;
}

}  // extern "C"
