// Double-double form: the modified Hermite integrators of Dittmann (2020) with
// every quantity and every operation in double-double arithmetic (dd.cuh, ~106
// bits), for few-body systems whose 8th-order (and higher) integration reaches
// the round-off of FP64 (Section 3.1, the 8th-order Kepler test; the
// Discussion's case for high-order schemes with extended precision).
//
// One step is the P(EC)^n shared step of the FP64 form: Taylor predictor
// (Section 3 intro), n times { O(N^2) evaluation of a^(0..p) (Section 3 intro),
// corrector: velocity by Eq. 6, then position by Eq. 7 with beta of Eq. 20 },
// then a^(p+1..2p-1) from the end-of-step Hermite interpolant (Eqs. 2-5).
// The state x, v, the derivative stack, the predicted trajectory, the pair
// terms and every sum are double-double; the corrector and interpolation
// constants are formed to 106 bits from exact rationals (hermite_consts_dd.cuh).
//
// Layout in device memory (each double-double is a double2 {hi, lo}):
//   x, v   N x 3          d   N x 2p x 3 (a^(0..2p-1))
//   tr     N x (P+1) x 3  trajectory fed to an evaluation (x, v, a, a-dot, ...)
//   part   S x N x (P+1) x 3  per-j-chunk (or per-distance) partial sums, added
//                         by the consumer in slot order, so results do not
//                         depend on scheduling.
// Kernels:
//   k_dd_pair_sym<P>  from 2048 bodies up: each unordered pair of bodies once,
//                     both bodies' terms from one evaluation, items of two
//                     64-body blocks, one partial-sum slot per (distance, side).
//   k_dd_pair<P, false>  one i per thread over one j-chunk, j records staged
//                     in shared memory; FP64-pipe bound (double-double costs
//                     about 20 FP64 operations per FP64 operation of the plain
//                     form).
//   k_dd_pair<P, true>   the same sums for the initialisation passes P = 7, 9,
//                     keeping only the two orders such a pass stores.
//   k_dd_predict<p>   one (body, component) per thread.
//   k_dd_reduce_slots<p>  adds the S partial sums in slot order, one thread
//                     per (body, order, component).
//   k_dd_correct<p>   one (body, component) per thread: corrects, and on the
//                     last pass commits the step and interpolates the higher
//                     derivatives.
//   k_dd_init_*       the explicit initial derivatives in passes of two orders.
//   k_dd_energy / k_dd_ecc   diagnostics (Appendix A) in double-double.
// Batched form (mh_dd_create_batch): many independent systems of up to 64
// bodies, each with its own dt.  k_dd_pair_sys gives system s one CTA holding
// its records in shared memory; the predictor and corrector read each body's
// dt through its system index; k_dd_energy_sys reduces each system's energy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "dd.cuh"
#include "hermite_consts_dd.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

constexpr int kDDThreads = 128;
constexpr int kDDJTile = 32;
constexpr int kDDTargetCtas = 152 * 8;   // evaluation grid: a few waves over the 152 SMs
constexpr int kDDMinJ = 1;               // fewest j per chunk: small systems spread one pair per thread
constexpr int kDDSysMax = 64;            // batched form: bodies per system (one CTA each)

__device__ __forceinline__ dd ld2(const double2 *p)
{
    const double2 v = *p;
    return dd(v.x, v.y);
}

__device__ __forceinline__ void st2(double2 *p, dd a) { *p = make_double2(a.hi, a.lo); }

__device__ __forceinline__ dd dot3(const dd *a, const dd *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// 1/y for a double-double y: the double reciprocal of y.hi and one Newton step
// with the residual 1 - y q formed in double-double.
__device__ __forceinline__ dd dd_inv(dd y)
{
    const double q = __drcp_rn(y.hi);
    const dd w = y * dd(q);
    const double e = __dsub_rn(__dsub_rn(1.0, w.hi), w.lo);
    return fast_two_sum(q, __dmul_rn(q, e));
}

// ---- constants (exact rationals to double-double) ----

template <int p>
struct DDTab;
#define MH_DD_TAB(P, KV, KX, E1, E0)                                                                     \
    template <>                                                                                          \
    struct DDTab<P> {                                                                                    \
        __device__ static dd kv(int k) { const ddc::Ratio r = KV(k); return dd_ratio(r.num, r.den); }     \
        __device__ static dd kx(int b, int k) { const ddc::Ratio r = KX(b, k); return dd_ratio(r.num, r.den); } \
        __device__ static dd e1(int n, int k) { const ddc::Ratio r = E1(n, k); return dd_ratio(r.num, r.den); } \
        __device__ static dd e0(int n, int k) { const ddc::Ratio r = E0(n, k); return dd_ratio(r.num, r.den); } \
    };
__host__ __device__ constexpr ddc::Ratio no_ratio(int, int) { return ddc::Ratio{0, 1}; }
MH_DD_TAB(1, ddc::kv1, ddc::kx1, no_ratio, no_ratio)
MH_DD_TAB(2, ddc::kv2, ddc::kx2, ddc::e1_2, ddc::e0_2)
MH_DD_TAB(3, ddc::kv3, ddc::kx3, ddc::e1_3, ddc::e0_3)
MH_DD_TAB(4, ddc::kv4, ddc::kx4, ddc::e1_4, ddc::e0_4)
MH_DD_TAB(5, ddc::kv5, ddc::kx5, ddc::e1_5, ddc::e0_5)
#undef MH_DD_TAB

__device__ __forceinline__ long long factorial_ll(int n)
{
    long long f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// The constants of every order, formed once per process by k_dd_consts (each
// a division pair, so forming them per thread would put ~50 FP64 divisions on
// every predictor and corrector thread) and read with warp-uniform indices.
constexpr int kDDMaxP = 5;
struct DDConsts {
    double2 kv[kDDMaxP + 1][kDDMaxP + 2];                 // [p][k]
    double2 kx[kDDMaxP + 1][2][kDDMaxP + 3];              // [p][beta_mode][k]
    double2 e1[kDDMaxP + 1][kDDMaxP][kDDMaxP + 2];        // [p][n - p - 1][k]
    double2 e0[kDDMaxP + 1][kDDMaxP][kDDMaxP + 2];
    double2 inv_fact[2 * kDDMaxP + 4];                   // 1/n!
};
__constant__ DDConsts c_ddc;
__device__ DDConsts g_ddc_stage;

template <int p>
__device__ void fill_consts(DDConsts &t)
{
    using Tab = DDTab<p>;
    for (int k = 0; k <= p; ++k) st2(&t.kv[p][k], Tab::kv(k));
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k <= p + 1; ++k) st2(&t.kx[p][b][k], Tab::kx(b, k));
    for (int n = p + 1; n < 2 * p; ++n)
        for (int k = 0; k <= p; ++k) {
            st2(&t.e1[p][n - p - 1][k], Tab::e1(n, k));
            st2(&t.e0[p][n - p - 1][k], Tab::e0(n, k));
        }
}

__global__ void k_dd_consts()
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fill_consts<1>(g_ddc_stage);
    fill_consts<2>(g_ddc_stage);
    fill_consts<3>(g_ddc_stage);
    fill_consts<4>(g_ddc_stage);
    fill_consts<5>(g_ddc_stage);
    for (int n = 0; n < 2 * kDDMaxP + 4; ++n) st2(&g_ddc_stage.inv_fact[n], dd_ratio(1, factorial_ll(n)));
}

__device__ __forceinline__ dd cget(const double2 &c) { return dd(c.x, c.y); }
__device__ __forceinline__ dd inv_fact_dd(int n) { return cget(c_ddc.inv_fact[n]); }

// ---- evaluation ----

// One pair's a^(0..P) of body i due to body j (Section 3 intro), added to acc:
// ti, tj the trajectory records x, v, a, ... (P + 1 vectors) of i and j.
template <int P>
__device__ __forceinline__ void dd_pair_full(const double2 *tj, const double2 *ti, double mj, dd eps2,
                                             double G, dd (&acc)[P + 1][3])
{
    dd r[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) r[k][c] = ld2(&tj[k * 3 + c]) - ld2(&ti[k * 3 + c]);
    const dd s = eps2 + (r[0][0] * r[0][0] + r[0][1] * r[0][1] + r[0][2] * r[0][2]);
    const dd y = rsqrt_dd(s);
    const dd sinv = y * y;
    const dd mS = two_prod(G, mj) * (sinv * y);
    pair_derivs<P, dd>(r, mS, sinv, acc);
}

// The initialisation passes with many derivatives (P = 7, 9: the 10th- and
// 12th-order starts) store only a^(P-1) and a^(P) (the lower orders are known).
// Holding r^(0..P), A^(0..P) and the sums of every order per pair would go far
// beyond the register file, so this form keeps the scalars q_k = s^(k)/s and
// tau_k (the recursion of pair_terms in pair_math.cuh), forms each r^(k) from
// the records when it is needed, and runs the A recursion one component at a
// time:  A^(n)_c = G m S r^(n)_c - sum_{k=1..n} C(n,k) tau_k A^(n-k)_c.
template <int P>
__device__ __forceinline__ void dd_pair_top2(const double2 *tj, const double2 *ti, double mj, dd eps2,
                                             double G, dd (&acc)[2][3])
{
    auto rk = [&](int k, int c) { return ld2(&tj[k * 3 + c]) - ld2(&ti[k * 3 + c]); };
    auto rdot = [&](int a, int b) { return rk(a, 0) * rk(b, 0) + rk(a, 1) * rk(b, 1) + rk(a, 2) * rk(b, 2); };
    const dd s = eps2 + rdot(0, 0);
    const dd y = rsqrt_dd(s);
    const dd sinv = y * y;
    const dd mS = two_prod(G, mj) * (sinv * y);
    dd q[P + 1], tau[P + 1];
#pragma unroll
    for (int k = 1; k <= P; ++k) {          // q_k = s^(k)/s, s^(k) = sum_j C(k,j) r^(j).r^(k-j)
        dd sk = dd(0.0);
#pragma unroll
        for (int j = 0; 2 * j <= k; ++j) sk += dd((2 * j == k) ? binom(k, j) : 2.0 * binom(k, j)) * rdot(j, k - j);
        q[k] = sk * sinv;
    }
    tau[0] = dd(1.0);
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        dd t = dd(1.5) * q[n];
#pragma unroll
        for (int j = 1; j <= n - 1; ++j) t += dd(1.5 * binom(n - 1, j - 1) - binom(n - 1, j)) * q[j] * tau[n - j];
        tau[n] = t;
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        dd A[P + 1];
#pragma unroll
        for (int n = 0; n <= P; ++n) {
            dd a = mS * rk(n, c);
#pragma unroll
            for (int k = 1; k <= n; ++k) a -= (dd(binom(n, k)) * tau[k]) * A[n - k];
            A[n] = a;
        }
        acc[0][c] += A[P - 1];
        acc[1][c] += A[P];
    }
}

// Sums of either form for body i over the records sj[0..n) (skipping jself),
// written to o: all orders, or (kTop2) orders P-1 and P at their places.
template <int P, bool kTop2>
__device__ __forceinline__ void dd_pair_sum(const double2 *sj, const double *smj, int n, int jself,
                                            const double2 *ti, dd eps2, double G, dd (&acc)[kTop2 ? 2 : P + 1][3])
{
    constexpr int R = (P + 1) * 3;
    for (int jj = 0; jj < n; ++jj) {
        if (jj == jself) continue;
        if constexpr (kTop2)
            dd_pair_top2<P>(sj + jj * R, ti, smj[jj], eps2, G, acc);
        else
            dd_pair_full<P>(sj + jj * R, ti, smj[jj], eps2, G, acc);
    }
}

template <int P, bool kTop2>
__device__ __forceinline__ void dd_store_sums(double2 *o, const dd (&acc)[kTop2 ? 2 : P + 1][3])
{
    constexpr int K0 = kTop2 ? P - 1 : 0;
#pragma unroll
    for (int k = 0; k < (kTop2 ? 2 : P + 1); ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) st2(&o[(K0 + k) * 3 + c], acc[k][c]);
}

// One system: part[split][i] = sum over j in chunk `split`, j != i.  Grid:
// (ceil(N / 128), S); j records staged in shared memory 32 at a time.
template <int P, bool kTop2>
__global__ void __launch_bounds__(kDDThreads)
k_dd_pair(const double2 *__restrict__ tr, const double *__restrict__ m, int N, double eps, double G,
          int jchunk, double2 *__restrict__ part)
{
    constexpr int R = (P + 1) * 3;
    __shared__ double2 sj[kDDJTile * R];
    __shared__ double sm[kDDJTile];
    const int i = blockIdx.x * kDDThreads + threadIdx.x;
    const int j0 = blockIdx.y * jchunk;
    const int j1 = min(N, j0 + jchunk);
    const bool live = i < N;
    const dd eps2 = two_prod(eps, eps);
    const double2 *ti = tr + (size_t)(live ? i : 0) * R;
    dd acc[kTop2 ? 2 : P + 1][3];
#pragma unroll
    for (int k = 0; k < (kTop2 ? 2 : P + 1); ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c] = dd(0.0);
    for (int jt = j0; jt < j1; jt += kDDJTile) {
        const int nt = min(kDDJTile, j1 - jt);
        __syncthreads();
        for (int q = threadIdx.x; q < nt * R; q += kDDThreads) sj[q] = tr[(size_t)jt * R + q];
        for (int q = threadIdx.x; q < nt; q += kDDThreads) sm[q] = m[jt + q];
        __syncthreads();
        if (live) dd_pair_sum<P, kTop2>(sj, sm, nt, i - jt, ti, eps2, G, acc);
    }
    if (live) dd_store_sums<P, kTop2>(part + ((size_t)blockIdx.y * N + i) * R, acc);
}

// Many independent systems (batched form): CTA s holds system s (at most
// kDDSysMax bodies, records off[s] .. off[s+1]-1) in shared memory; warp w
// sums bodies 32 w .. 32 w + m - 1 of the system (m <= 32) over the whole
// system, into a single partial-sum slot.  Where m leaves lanes idle (systems
// below 32 bodies, or the second warp of one with 33 .. 64), each body gets a
// group of g lanes (g the largest power of two with g m <= 32): lane l takes
// body l / g over the sources j = l mod g, l mod g + g, ..., and the g partial
// sums meet in a fixed xor-shuffle tree of double-word additions.  A warp
// instruction costs the FP64 pipe the same with 3 lanes live as with 32, so
// the groups cut the pair iterations of a system of m < 32 bodies per warp by
// g, for log2(g) tree levels; each body's summation order depends on the
// system alone.
template <int P, bool kTop2>
__global__ void __launch_bounds__(kDDSysMax)
k_dd_pair_sys(const double2 *__restrict__ tr, const double *__restrict__ m, const int64_t *__restrict__ off,
              double eps, double G, double2 *__restrict__ part)
{
    constexpr int R = (P + 1) * 3;
    constexpr int NA = kTop2 ? 2 : P + 1;
    __shared__ double2 sj[kDDSysMax * R];
    __shared__ double sm[kDDSysMax];
    const int64_t b0 = off[blockIdx.x];
    const int n = (int)(off[blockIdx.x + 1] - b0);
    for (int q = threadIdx.x; q < n * R; q += kDDSysMax) sj[q] = tr[(size_t)b0 * R + q];
    for (int q = threadIdx.x; q < n; q += kDDSysMax) sm[q] = m[b0 + q];
    __syncthreads();
    const int lane = threadIdx.x & 31, base = threadIdx.x & ~31;
    if (base >= n) return;                          // the whole warp
    const int mb = min(32, n - base);
    int g = 1;
    while (2 * g * mb <= 32) g *= 2;
    const int k0 = lane / g, sub = lane - k0 * g;
    const int i = base + (k0 < mb ? k0 : 0);        // lanes past the groups repeat body base
    const dd eps2 = two_prod(eps, eps);
    dd acc[NA][3];
#pragma unroll
    for (int k = 0; k < NA; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c] = dd(0.0);
    const double2 *ti = sj + i * R;
    for (int j = sub; j < n; j += g) {
        if (j == i) continue;
        if constexpr (kTop2)
            dd_pair_top2<P>(sj + j * R, ti, sm[j], eps2, G, acc);
        else
            dd_pair_full<P>(sj + j * R, ti, sm[j], eps2, G, acc);
    }
    for (int o = 1; o < g; o *= 2)
#pragma unroll
        for (int k = 0; k < NA; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double h = __shfl_xor_sync(0xffffffffu, acc[k][c].hi, o);
                const double l = __shfl_xor_sync(0xffffffffu, acc[k][c].lo, o);
                acc[k][c] = acc[k][c] + dd(h, l);
            }
    if (sub == 0 && k0 < mb) dd_store_sums<P, kTop2>(part + (size_t)(b0 + i) * R, acc);
}

// ---- pair-symmetric evaluation ----
//
// Each scaled pair term B_k (pair_math.cuh) is odd under i <-> j and the factor
// S = s^-3/2 is even, so one evaluation of a pair gives both bodies' terms:
// body i gets m_j (G S B_k) and body j gets -m_i (G S B_k).  Bodies form blocks
// of kDDSymB = 32 W (W warps; nB blocks, the last one ragged).  An item is one
// block pair (I, J = I + b mod nB): b = 1 .. Dfull for every row I (Dfull =
// (nB - 1) / 2), and, when nB is even, the half distance b = nB / 2 for the
// rows I < nB / 2 only, so that every unordered block pair is one item; b = 0
// is the block with itself.  The CTA keeps block J's records and running
// j-side sums in shared memory (row-major by record element, so the 32 lanes
// of a ring step hit distinct banks); thread t owns body I kDDSymB + t.  Warp
// w runs 32-step rings over j-subtile q = (w + phase) mod W, lane l pairing
// with j = 32 q + (l + s) mod 32: within a phase no two warps share a subtile
// and no two lanes a j, so the j-side sums are read, added to and written back
// without atomics, in an order fixed by (phase, step).  A diagonal item takes
// every unordered pair once by the same rings: within the own subtile the ring
// distances 1 .. 16 (16 on lanes 0 .. 15 only), and subtile pairs (w, w + ph)
// for ph < W/2, plus ph = W/2 for w < W/2.  A ring whose lanes are all past N
// (the ragged last block) is skipped.
//
// Output: item (I, b) writes its i-side sums to slot b and its j-side sums to
// slot Dmax + b (Dmax = nB / 2), except the half distance, whose j-side bodies
// (blocks >= nB / 2) take slot b, the one their own i-side leaves empty; a
// diagonal item adds its j-side sums to its i-side ones (in that order) into
// slot 0.  Every body of every slot 0 .. nB - 1 is then written exactly once,
// and the consumer adds the slots in slot order: deterministic results.
// The sums use the sloppy double-word addition (dd.cuh: error ~u^2 of the
// summed magnitudes, the same order as the terms' own rounding) and raw
// products by the masses: ~950 FP64 operations per pair interaction at P = 3,
// against ~1800 for k_dd_pair.  Two warps per block: items of 64 x 64 pairs
// are small enough that 152 SMs finish together (with 128-body blocks, 3.5
// items per SM at 4096 bodies left SMs idle for the last item).  Slots take
// nB N (P + 1) 3 double-words (75 MB at N = 4096, P = 3); the planner keeps
// them within kDDSymMaxBytes.
constexpr int kDDSymW = 2;
constexpr int kDDSymB = 32 * kDDSymW;

struct DDSymItem {
    int I, b;
};

__host__ __device__ __forceinline__ DDSymItem dd_sym_item(int t, int nB)
{
    const int Dfull = (nB - 1) / 2;
    DDSymItem it;
    if (t < nB * Dfull) {                       // full distances, largest work first
        it.b = 1 + t / nB;
        it.I = t - (it.b - 1) * nB;
    } else if ((nB & 1) == 0 && t < nB * Dfull + nB / 2) {   // half distance, rows < nB / 2
        it.b = nB / 2;
        it.I = t - nB * Dfull;
    } else {                                    // diagonal blocks (half the pairs) last
        it.b = 0;
        it.I = t - nB * Dfull - ((nB & 1) ? 0 : nB / 2);
    }
    return it;
}

__host__ __device__ __forceinline__ int dd_sym_items(int nB) { return nB * ((nB - 1) / 2) + ((nB & 1) ? 0 : nB / 2) + nB; }

// Ring steps [s0, s1) of warp w in phase ph (over subtile (w + ph) mod W), and
// whether the pair of a lane at step s counts: all 32 steps off the diagonal;
// on it, the rules above.
__host__ __device__ __forceinline__ void dd_sym_steps(bool diag, int ph, int w, int &s0, int &s1)
{
    s0 = 0;
    s1 = 32;
    if (diag) {
        if (ph == 0) { s0 = 1; s1 = 17; }
        else if (!(2 * ph < kDDSymW || (2 * ph == kDDSymW && w < kDDSymW / 2))) s1 = 0;
    }
}

__host__ __device__ __forceinline__ bool dd_sym_take(bool diag, int ph, int s, int lane)
{
    return !(diag && ph == 0 && s == 16 && lane >= 16);
}

template <int P>
__host__ __device__ constexpr size_t dd_sym_smem() { return (size_t)kDDSymB * (2 * (P + 1) * 3 * sizeof(double2) + sizeof(double)); }

template <int P>
__global__ void __launch_bounds__(kDDSymB, 8 / kDDSymW)
k_dd_pair_sym(const double2 *__restrict__ tr, const double *__restrict__ m, int N, int nB, double eps, double G,
              double2 *__restrict__ part)
{
    constexpr int R = (P + 1) * 3;
    extern __shared__ double2 dd_sym_sh[];
    double2 *sj = dd_sym_sh;                        // [R][kDDSymB] records of block J
    double2 *ja = sj + R * kDDSymB;                 // [R][kDDSymB] j-side sums
    double *sm = (double *)(ja + R * kDDSymB);      // [kDDSymB] masses of block J (0 past N)
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const DDSymItem it = dd_sym_item(blockIdx.x, nB);
    const bool diag = it.b == 0;
    const int J = diag ? it.I : (it.I + it.b) % nB;
    const int i = it.I * kDDSymB + t, j0 = J * kDDSymB;
    for (int q = t; q < R * kDDSymB; q += kDDSymB) {
        const int jj = q / R, e = q - jj * R;       // coalesced over the AoS rows of the block
        const int j = j0 + jj;
        sj[e * kDDSymB + jj] = j < N ? tr[(size_t)j * R + e] : make_double2(0.0, 0.0);
        ja[e * kDDSymB + jj] = make_double2(0.0, 0.0);
    }
    sm[t] = j0 + t < N ? m[j0 + t] : 0.0;
    const bool ilive = i < N;
    const double mi = ilive ? m[i] : 0.0;
    dd ri[P + 1][3], acc[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ri[k][c] = ilive ? ld2(&tr[(size_t)i * R + k * 3 + c]) : dd(0.0);
            acc[k][c] = dd(0.0);
        }
    const dd eps2 = two_prod(eps, eps);
    __syncthreads();
    for (int ph = 0; ph < kDDSymW; ++ph) {
        const int q = (w + ph) % kDDSymW;
        int s0, s1;
        dd_sym_steps(diag, ph, w, s0, s1);
        if (it.I * kDDSymB + 32 * w >= N || j0 + 32 * q >= N) s1 = s0;   // every lane past N
        for (int s = s0; s < s1; ++s) {
            const int jj = q * 32 + ((lane + s) & 31);
            const bool live = ilive && j0 + jj < N && dd_sym_take(diag, ph, s, lane);
            dd r[P + 1][3];
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) r[k][c] = ld2(&sj[(k * 3 + c) * kDDSymB + jj]) - ri[k][c];
            dd s2 = eps2 + (r[0][0] * r[0][0] + r[0][1] * r[0][1] + r[0][2] * r[0][2]);
            s2 = live ? s2 : dd(1.0);
            const double mj = live ? sm[jj] : 0.0, mi_live = live ? mi : 0.0;
            const dd y = rsqrt_dd(s2);
            const dd sinv = y * y;
            const dd GS = mul_d(sinv * y, G);
            pair_odd_terms<P, dd>(r, sinv, [&](int k, int c, dd B) {
                const dd sb = GS * B;
                acc[k][c] = add_sloppy(acc[k][c], mul_d_raw(sb, mj));
                double2 *pj = &ja[(k * 3 + c) * kDDSymB + jj];
                st2(pj, add_sloppy(ld2(pj), mul_d_raw(sb, -mi_live)));
            });
            __syncwarp();
        }
        __syncthreads();
    }
    const int slot_i = it.b;
    const int Dmax = nB / 2;
    if (diag) {
        if (ilive)
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    st2(&part[(size_t)i * R + k * 3 + c], acc[k][c] + ld2(&ja[(k * 3 + c) * kDDSymB + t]));
        return;
    }
    if (ilive) dd_store_sums<P, false>(part + ((size_t)slot_i * N + i) * R, acc);
    const int slot_j = ((nB & 1) == 0 && it.b == Dmax) ? it.b : Dmax + it.b;
    const int j = j0 + t;
    if (j < N)
#pragma unroll
        for (int e = 0; e < R; ++e) part[((size_t)slot_j * N + j) * R + e] = ja[e * kDDSymB + t];
}

// Adds the S partial-sum slots of a^(0..p) in slot order into slot 0, one
// thread per (body, order, component), so that the corrector reads one slot.
// (A serial sum of S slots for all p + 1 orders in every corrector thread is a
// chain of S (p + 1) double-double additions, each ~20 FP64 instructions of
// ~64 cycles per warp on GB300: the latency of small systems.)
template <int p>
__global__ void __launch_bounds__(kDDThreads)
k_dd_reduce_slots(double2 *__restrict__ part, int S, int N)
{
    constexpr int R = (p + 1) * 3;
    const int64_t t = (int64_t)blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= (int64_t)N * R) return;
    dd s = ld2(&part[t]);
    for (int q = 1; q < S; ++q) s += ld2(&part[(size_t)q * N * R + t]);
    st2(&part[t], s);
}

// The same for any record width: nt = N R elements per slot.
__global__ void __launch_bounds__(kDDThreads)
k_dd_add_slots(double2 *__restrict__ part, int S, int64_t nt)
{
    const int64_t t = (int64_t)blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= nt) return;
    dd s = ld2(&part[t]);
    for (int q = 1; q < S; ++q) s += ld2(&part[(size_t)q * nt + t]);
    st2(&part[t], s);
}

// ---- predictor ----

// Taylor series of x, v and a^(0..p-2) to t0 + dt (Section 3 intro, with every
// derivative the step holds), written as the trajectory record of the first
// evaluation.  One thread per (body, component).
template <int p>
__global__ void __launch_bounds__(kDDThreads)
k_dd_predict(const double2 *__restrict__ x, const double2 *__restrict__ v, const double2 *__restrict__ d,
             int N, double dt0, const double *__restrict__ dts, const int *__restrict__ sys,
             double2 *__restrict__ tr)
{
    constexpr int K = 2 * p, R = (p + 1) * 3;
    const int t = blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= 3 * N) return;
    const int i = t / 3, c = t - 3 * i;
    const double dt = dts ? dts[sys[i]] : dt0;      // batched form: each system its own step
    dd a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = ld2(&d[((size_t)i * K + k) * 3 + c]);
    dd sx = dd(0.0), sv = dd(0.0);
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        sx = mul_d(sx, dt) + a[k] * inv_fact_dd(k + 2);
        sv = mul_d(sv, dt) + a[k] * inv_fact_dd(k + 1);
    }
    const dd x0 = ld2(&x[(size_t)i * 3 + c]), v0 = ld2(&v[(size_t)i * 3 + c]);
    double2 *o = tr + (size_t)i * R;
    st2(&o[c], mul_d(mul_d(sx, dt) + v0, dt) + x0);
    st2(&o[3 + c], mul_d(sv, dt) + v0);
#pragma unroll
    for (int q = 0; q + 2 <= p; ++q) {
        dd sa = dd(0.0);
#pragma unroll
        for (int k = K - 1; k >= q; --k) sa = mul_d(sa, dt) + a[k] * inv_fact_dd(k - q);
        st2(&o[(q + 2) * 3 + c], sa);
    }
}

// ---- corrector ----

// One correction pass (Eqs. 6, 7 in dt-power form: velocity first, then the
// position with the new velocity).  a^(0..p) at t1 are the S partial sums added
// in chunk order.  Not last: writes the next evaluation's trajectory record
// (x1, v1 and a^(0..p-2) of this evaluation).  Last: commits x, v and
// a^(0..p), and a^(p+1..2p-1) from the Hermite interpolant; flags a non-finite
// state.
template <int p, bool kLast>
__global__ void __launch_bounds__(kDDThreads)
k_dd_correct(double2 *__restrict__ x, double2 *__restrict__ v, double2 *__restrict__ d,
             const double2 *__restrict__ part, int S, int N, double dt0, const double *__restrict__ dts,
             const int *__restrict__ sys, int bm, double2 *__restrict__ tr, int *__restrict__ flag)
{
    constexpr int K = 2 * p, R = (p + 1) * 3;
    const int t = blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= 3 * N) return;
    const int i = t / 3, c = t - 3 * i;
    const double dt = dts ? dts[sys[i]] : dt0;
    dd a1[p + 1], a0[p + 1];
#pragma unroll
    for (int k = 0; k <= p; ++k) {
        dd s = dd(0.0);
        for (int q = 0; q < S; ++q) s += ld2(&part[((size_t)q * N + i) * R + k * 3 + c]);
        a1[k] = s;
        a0[k] = ld2(&d[((size_t)i * K + k) * 3 + c]);
    }
    const dd x0 = ld2(&x[(size_t)i * 3 + c]), v0 = ld2(&v[(size_t)i * 3 + c]);
    // velocity: sum_k kv(k) (a1^(k) + (-1)^k a0^(k)) dt^(k+1)
    dd sv = dd(0.0);
#pragma unroll
    for (int k = p; k >= 0; --k) {
        const dd f = (k & 1) ? a1[k] - a0[k] : a1[k] + a0[k];
        sv = mul_d(sv, dt) + cget(c_ddc.kv[p][k]) * f;
    }
    const dd vn = mul_d(sv, dt) + v0;
    // position: kx(0) (v1 + v0) dt + sum_{k>=1} kx(k) (a1^(k-1) +- a0^(k-1)) dt^(k+1)
    dd sx = dd(0.0);
#pragma unroll
    for (int k = p + 1; k >= 1; --k) {
        const dd f = (k & 1) ? a1[k - 1] - a0[k - 1] : a1[k - 1] + a0[k - 1];
        sx = mul_d(sx, dt) + cget(c_ddc.kx[p][bm][k]) * f;
    }
    sx = mul_d(sx, dt) + cget(c_ddc.kx[p][bm][0]) * (vn + v0);
    const dd xn = mul_d(sx, dt) + x0;
    if constexpr (!kLast) {
        double2 *o = tr + (size_t)i * R;
        st2(&o[c], xn);
        st2(&o[3 + c], vn);
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) st2(&o[(q + 2) * 3 + c], a1[q]);
    } else {
        st2(&x[(size_t)i * 3 + c], xn);
        st2(&v[(size_t)i * 3 + c], vn);
        if (!dd_isfinite(xn) || !dd_isfinite(vn)) *flag = 1;
#pragma unroll
        for (int k = 0; k <= p; ++k) st2(&d[((size_t)i * K + k) * 3 + c], a1[k]);
        if constexpr (p >= 2) {
            // a^(n)(t1) = sum_k (e1(n,k) a1^(k) + e0(n,k) a0^(k)) dt^(k-n)
            const dd rdt = dd_recip(dt);
#pragma unroll
            for (int n = p + 1; n < K; ++n) {
                dd s = dd(0.0);
#pragma unroll
                for (int k = p; k >= 0; --k)
                    s = mul_d(s, dt) + (cget(c_ddc.e1[p][n - p - 1][k]) * a1[k] + cget(c_ddc.e0[p][n - p - 1][k]) * a0[k]);
#pragma unroll
                for (int e = 0; e < n; ++e) s = s * rdt;
                st2(&d[((size_t)i * K + n) * 3 + c], s);
            }
        }
    }
}

// ---- initialisation (Section 3 intro) ----

// Trajectory records x, v, a^(0..have-1) (R = have + 2 vectors per body).
__global__ void k_dd_init_tr(const double2 *__restrict__ x, const double2 *__restrict__ v,
                             const double2 *__restrict__ d, int N, int K, int have, double2 *__restrict__ tr)
{
    const int R = (have + 2) * 3;
    const int64_t t = (int64_t)blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= (int64_t)N * R) return;
    const int i = (int)(t / R), q = (int)(t - (int64_t)i * R);
    const int k = q / 3, c = q - 3 * k;
    tr[t] = k == 0 ? x[(size_t)i * 3 + c] : k == 1 ? v[(size_t)i * 3 + c] : d[((size_t)i * K + k - 2) * 3 + c];
}

// d[i][n] = sum over the S chunks, n = have .. min(P, K-1).
__global__ void k_dd_init_store(const double2 *__restrict__ part, int S, int N, int P, int K, int have,
                                double2 *__restrict__ d)
{
    const int R = (P + 1) * 3;
    const int nn = min(P, K - 1) - have + 1;
    const int64_t t = (int64_t)blockIdx.x * kDDThreads + threadIdx.x;
    if (t >= (int64_t)N * nn * 3) return;
    const int i = (int)(t / (nn * 3)), q = (int)(t - (int64_t)i * nn * 3);
    const int n = have + q / 3, c = q % 3;
    dd s = dd(0.0);
    for (int u = 0; u < S; ++u) s += ld2(&part[((size_t)u * N + i) * R + n * 3 + c]);
    st2(&d[((size_t)i * K + n) * 3 + c], s);
}

// ---- diagnostics (Appendix A) ----

// Per-CTA partial energies: sum over the CTA's bodies i of m_i |v_i|^2 / 2 -
// sum_{j > i} G m_i m_j / sqrt(r_ij^2 + eps^2), reduced by a fixed tree.
__global__ void __launch_bounds__(kDDThreads)
k_dd_energy(const double *__restrict__ m, const double2 *__restrict__ x, const double2 *__restrict__ v,
            int N, double eps, double G, double2 *__restrict__ bpart)
{
    __shared__ double2 sh[kDDThreads];
    const int i = blockIdx.x * kDDThreads + threadIdx.x;
    dd e = dd(0.0);
    if (i < N) {
        dd xi[3], vi[3];
        for (int c = 0; c < 3; ++c) { xi[c] = ld2(&x[(size_t)i * 3 + c]); vi[c] = ld2(&v[(size_t)i * 3 + c]); }
        const dd eps2 = two_prod(eps, eps);
        dd pot = dd(0.0);
        for (int j = i + 1; j < N; ++j) {
            dd r[3];
            for (int c = 0; c < 3; ++c) r[c] = ld2(&x[(size_t)j * 3 + c]) - xi[c];
            pot += dd(m[j]) * rsqrt_dd(eps2 + dot3(r, r));
        }
        e = mul_d(mul_d(dot3(vi, vi), m[i]), 0.5) - pot * two_prod(G, m[i]);
    }
    st2(&sh[threadIdx.x], e);
    __syncthreads();
    for (int s = kDDThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) st2(&sh[threadIdx.x], ld2(&sh[threadIdx.x]) + ld2(&sh[threadIdx.x + s]));
        __syncthreads();
    }
    if (threadIdx.x == 0) bpart[blockIdx.x] = sh[0];
}

// Batched form: the energy of system s (CTA s), reduced over its bodies by a
// fixed tree.
__global__ void __launch_bounds__(kDDSysMax)
k_dd_energy_sys(const double *__restrict__ m, const double2 *__restrict__ x, const double2 *__restrict__ v,
                const int64_t *__restrict__ off, double eps, double G, double2 *__restrict__ out)
{
    __shared__ double2 sh[kDDSysMax];
    const int64_t b0 = off[blockIdx.x];
    const int n = (int)(off[blockIdx.x + 1] - b0);
    const int t = threadIdx.x;
    dd e = dd(0.0);
    if (t < n) {
        const int64_t i = b0 + t;
        dd xi[3], vi[3];
        for (int c = 0; c < 3; ++c) { xi[c] = ld2(&x[i * 3 + c]); vi[c] = ld2(&v[i * 3 + c]); }
        const dd eps2 = two_prod(eps, eps);
        dd pot = dd(0.0);
        for (int64_t j = i + 1; j < b0 + n; ++j) {
            dd r[3];
            for (int c = 0; c < 3; ++c) r[c] = ld2(&x[j * 3 + c]) - xi[c];
            pot += dd(m[j]) * rsqrt_dd(eps2 + dot3(r, r));
        }
        e = mul_d(mul_d(dot3(vi, vi), m[i]), 0.5) - pot * two_prod(G, m[i]);
    }
    st2(&sh[t], e);
    __syncthreads();
    for (int h = kDDSysMax / 2; h > 0; h >>= 1) {
        if (t < h) st2(&sh[t], ld2(&sh[t]) + ld2(&sh[t + h]));
        __syncthreads();
    }
    if (t == 0) out[blockIdx.x] = sh[0];
}

__global__ void k_dd_sum(const double2 *__restrict__ bpart, int nb, double2 *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    dd s = dd(0.0);
    for (int b = 0; b < nb; ++b) s += ld2(&bpart[b]);
    st2(out, s);
}

// Eccentricity vectors about body `central` (Eq. A1): mu e = (|v|^2 - mu/|r|) r
// - (r.v) v with r, v relative to the central body and mu = G (m_c + m_i).
__global__ void k_dd_ecc(const double *__restrict__ m, const double2 *__restrict__ x,
                         const double2 *__restrict__ v, int N, double G, int central, double2 *__restrict__ e)
{
    const int i = blockIdx.x * kDDThreads + threadIdx.x;
    if (i >= N) return;
    if (i == central) {
        for (int c = 0; c < 3; ++c) e[(size_t)i * 3 + c] = make_double2(0.0, 0.0);
        return;
    }
    dd r[3], u[3];
    for (int c = 0; c < 3; ++c) {
        r[c] = ld2(&x[(size_t)i * 3 + c]) - ld2(&x[(size_t)central * 3 + c]);
        u[c] = ld2(&v[(size_t)i * 3 + c]) - ld2(&v[(size_t)central * 3 + c]);
    }
    const dd mu = mul_d(two_sum(m[central], m[i]), G);
    const dd w = dot3(u, u) - mu * rsqrt_dd(dot3(r, r));
    const dd rv = dot3(r, u);
    const dd rmu = dd_inv(mu);
    for (int c = 0; c < 3; ++c) st2(&e[(size_t)i * 3 + c], (w * r[c] - rv * u[c]) * rmu);
}

// ---- launch helpers ----

// An evaluation's grid: ordered pairs (iblocks x S j-chunks of jchunk bodies)
// or, when sym, the pair-symmetric items over nB blocks (S = nB slots).
struct DDPlan {
    int iblocks = 0, S = 1, jchunk = 0;
    bool sym = false;
    int nB = 0;
};

constexpr int kDDSymMinN = 2048;                         // automatic choice: from 16 blocks up
constexpr size_t kDDSymMaxBytes = (size_t)4 << 30;        // partial-sum slots of the symmetric kernel

// Whether an evaluation of N bodies with records of R double-words uses the
// pair-symmetric kernel (a simulation sizes its slots for the widest
// initialisation record, R = 6p): mode 0 never, 2 whenever the slots fit, 1
// from kDDSymMinN bodies up (below, the ordered kernel spreads the pairs over
// more SMs).
bool dd_use_sym(int N, int R, int mode)
{
    if (mode == 0) return false;
    const size_t nB = (size_t)((N + kDDSymB - 1) / kDDSymB);
    if (nB * (size_t)N * (size_t)R * sizeof(double2) > kDDSymMaxBytes) return false;
    return mode == 2 || N >= kDDSymMinN;
}

DDPlan dd_plan(int N, bool sym = false)
{
    DDPlan pl;
    if (sym) {
        pl.sym = true;
        pl.nB = (N + kDDSymB - 1) / kDDSymB;
        pl.S = pl.nB;
        return pl;
    }
    pl.iblocks = (N + kDDThreads - 1) / kDDThreads;
    int S = std::max(1, std::min((N + kDDMinJ - 1) / kDDMinJ, kDDTargetCtas / pl.iblocks));
    pl.jchunk = (N + S - 1) / S;
    pl.S = (N + pl.jchunk - 1) / pl.jchunk;
    return pl;
}

// Opens the dynamic shared memory of the symmetric kernels (set before any
// launch or capture; idempotent).
int dd_sym_attrs()
{
    MH_CUDA(cudaFuncSetAttribute(k_dd_pair_sym<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sym_smem<1>()));
    MH_CUDA(cudaFuncSetAttribute(k_dd_pair_sym<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sym_smem<2>()));
    MH_CUDA(cudaFuncSetAttribute(k_dd_pair_sym<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sym_smem<3>()));
    MH_CUDA(cudaFuncSetAttribute(k_dd_pair_sym<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sym_smem<4>()));
    MH_CUDA(cudaFuncSetAttribute(k_dd_pair_sym<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sym_smem<5>()));
    return MH_OK;
}

// Batched form on the device: system offsets, the system of every body, and
// the per-system steps.
struct DDBatchDev {
    const int64_t *off = nullptr;
    const int *sys = nullptr;
    const double *dts = nullptr;
    int S = 0;
};

template <int P, bool kTop2>
void launch_pair_kernel(const double2 *tr, const double *m, int N, double eps, double G, const DDPlan &pl,
                        double2 *part, cudaStream_t st, const DDBatchDev *b)
{
    if (b)
        k_dd_pair_sys<P, kTop2><<<b->S, kDDSysMax, 0, st>>>(tr, m, b->off, eps, G, part);
    else if constexpr (!kTop2 && P <= kDDMaxP)
        if (pl.sym)
            k_dd_pair_sym<P><<<dd_sym_items(pl.nB), kDDSymB, dd_sym_smem<P>(), st>>>(tr, m, N, pl.nB, eps, G, part);
        else
            k_dd_pair<P, kTop2><<<dim3(pl.iblocks, pl.S), kDDThreads, 0, st>>>(tr, m, N, eps, G, pl.jchunk, part);
    else
        k_dd_pair<P, kTop2><<<dim3(pl.iblocks, pl.S), kDDThreads, 0, st>>>(tr, m, N, eps, G, pl.jchunk, part);
}

int launch_dd_pair(int P, const double2 *tr, const double *m, int N, double eps, double G, const DDPlan &pl,
                   double2 *part, cudaStream_t st, const DDBatchDev *b)
{
    switch (P) {
        case 1: launch_pair_kernel<1, false>(tr, m, N, eps, G, pl, part, st, b); break;
        case 2: launch_pair_kernel<2, false>(tr, m, N, eps, G, pl, part, st, b); break;
        case 3: launch_pair_kernel<3, false>(tr, m, N, eps, G, pl, part, st, b); break;
        case 4: launch_pair_kernel<4, false>(tr, m, N, eps, G, pl, part, st, b); break;
        case 5: launch_pair_kernel<5, false>(tr, m, N, eps, G, pl, part, st, b); break;
        case 7: launch_pair_kernel<7, true>(tr, m, N, eps, G, pl, part, st, b); break;
        case 9: launch_pair_kernel<9, true>(tr, m, N, eps, G, pl, part, st, b); break;
        default: set_error("double-double evaluation: unsupported derivative count"); return MH_EINVAL;
    }
    MH_LAUNCHED("k_dd_pair");
    return MH_OK;
}

template <int p>
int launch_dd_step_p(double2 *x, double2 *v, double2 *d, double2 *tr, double2 *part, const double *m, int N,
                     double eps, double G, int bm, double dt, int n_iter, int *flag, cudaStream_t st,
                     const DDBatchDev *b, bool sym)
{
    const DDPlan pl = dd_plan(N, sym);
    const bool reduce = !b && pl.S > 1;
    const int slots = 1;                       // the corrector reads slot 0 (pre-summed when S > 1)
    const double *dts = b ? b->dts : nullptr;
    const int *sys = b ? b->sys : nullptr;
    const int nb = (3 * N + kDDThreads - 1) / kDDThreads;
    const int nr = (int)(((int64_t)N * (p + 1) * 3 + kDDThreads - 1) / kDDThreads);
    k_dd_predict<p><<<nb, kDDThreads, 0, st>>>(x, v, d, N, dt, dts, sys, tr);
    MH_LAUNCHED("k_dd_predict");
    for (int it = 0; it < n_iter; ++it) {
        if (int rc = launch_dd_pair(p, tr, m, N, eps, G, pl, part, st, b)) return rc;
        if (reduce) {
            k_dd_reduce_slots<p><<<nr, kDDThreads, 0, st>>>(part, pl.S, N);
            MH_LAUNCHED("k_dd_reduce_slots");
        }
        if (it + 1 < n_iter)
            k_dd_correct<p, false><<<nb, kDDThreads, 0, st>>>(x, v, d, part, slots, N, dt, dts, sys, bm, tr, flag);
        else
            k_dd_correct<p, true><<<nb, kDDThreads, 0, st>>>(x, v, d, part, slots, N, dt, dts, sys, bm, tr, flag);
        MH_LAUNCHED("k_dd_correct");
    }
    return MH_OK;
}

// host double-double add of a double (the simulation time)
void host_add(double &hi, double &lo, double b)
{
    const double s = hi + b;
    const double bv = s - hi;
    const double t = (hi - (s - bv)) + (b - bv);
    const double l = lo + t;
    hi = s + l;
    lo = l - (hi - s);
}

}  // namespace

}  // namespace mh

using namespace mh;

struct mh_dd {
    int64_t N = 0;
    int p = 0, order = 0, bm = 0;
    bool sym = false;               // single system: pair-symmetric evaluation (dd_use_sym)
    double eps = 0.0, G = 1.0;
    double t_hi = 0.0, t_lo = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *m = nullptr;
    double2 *x = nullptr, *v = nullptr, *d = nullptr, *tr = nullptr, *part = nullptr, *diag = nullptr;
    int *flag = nullptr;
    // batched form (S > 0): system offsets, system of each body, per-system steps
    int64_t S = 0;
    int64_t *off = nullptr;
    int *sys = nullptr;
    double *dts = nullptr;
    int64_t batch_steps = 0;
    double batch_pairs = 0.0;     // sum over systems of n_s (n_s - 1)
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int graph_n = 0;
    mh_counters ctr{};

    DDBatchDev batch() const
    {
        DDBatchDev b;
        b.off = off;
        b.sys = sys;
        b.dts = dts;
        b.S = (int)S;
        return b;
    }
};

namespace {

int dd_free(mh_dd *s)
{
    if (!s) return MH_OK;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    cudaFree(s->m); cudaFree(s->x); cudaFree(s->v); cudaFree(s->d);
    cudaFree(s->tr); cudaFree(s->part); cudaFree(s->diag); cudaFree(s->flag);
    cudaFree(s->off); cudaFree(s->sys); cudaFree(s->dts);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return MH_OK;
}

int dd_check(const mh_dd *s, const char *fn)
{
    if (!s) {
        set_error(std::string(fn) + ": handle is NULL");
        return MH_EINVAL;
    }
    return MH_OK;
}

// Forms the constant table (k_dd_consts) and copies it to constant memory, once
// per process.
int dd_consts_once(cudaStream_t st)
{
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return MH_OK;
    k_dd_consts<<<1, 32, 0, st>>>();
    MH_LAUNCHED("k_dd_consts");
    void *stage = nullptr;
    MH_CUDA(cudaGetSymbolAddress(&stage, g_ddc_stage));
    MH_CUDA(cudaMemcpyToSymbolAsync(c_ddc, stage, sizeof(DDConsts), 0, cudaMemcpyDeviceToDevice, st));
    MH_CUDA(cudaStreamSynchronize(st));
    done = true;
    return MH_OK;
}

int dd_initialise(mh_dd *s)
{
    const int N = (int)s->N, K = 2 * s->p;
    const DDBatchDev b = s->batch();
    const DDBatchDev *bp = s->S ? &b : nullptr;
    for (int have = 0; have < K; have += 2) {
        const int P = have + 1;
        const DDPlan pl = dd_plan(N, s->sym && P <= kDDMaxP);
        const int slots = s->S ? 1 : pl.S;
        const int64_t nt = (int64_t)N * (have + 2) * 3;
        k_dd_init_tr<<<(unsigned)((nt + kDDThreads - 1) / kDDThreads), kDDThreads, 0, s->stream>>>(
            s->x, s->v, s->d, N, K, have, s->tr);
        MH_LAUNCHED("k_dd_init_tr");
        if (int rc = launch_dd_pair(P, s->tr, s->m, N, s->eps, s->G, pl, s->part, s->stream, bp)) return rc;
        const int nn = std::min(P, K - 1) - have + 1;
        const int64_t ns = (int64_t)N * nn * 3;
        k_dd_init_store<<<(unsigned)((ns + kDDThreads - 1) / kDDThreads), kDDThreads, 0, s->stream>>>(
            s->part, slots, N, P, K, have, s->d);
        MH_LAUNCHED("k_dd_init_store");
        s->ctr.kernel_launches += 3;
    }
    return MH_OK;
}

int dd_step_once(mh_dd *s, double dt, int n_iter)
{
    const int N = (int)s->N;
    const DDBatchDev b = s->batch();
    const DDBatchDev *bp = s->S ? &b : nullptr;
    switch (s->p) {
        case 1: return launch_dd_step_p<1>(s->x, s->v, s->d, s->tr, s->part, s->m, N, s->eps, s->G, s->bm, dt, n_iter, s->flag, s->stream, bp, s->sym);
        case 2: return launch_dd_step_p<2>(s->x, s->v, s->d, s->tr, s->part, s->m, N, s->eps, s->G, s->bm, dt, n_iter, s->flag, s->stream, bp, s->sym);
        case 3: return launch_dd_step_p<3>(s->x, s->v, s->d, s->tr, s->part, s->m, N, s->eps, s->G, s->bm, dt, n_iter, s->flag, s->stream, bp, s->sym);
        case 4: return launch_dd_step_p<4>(s->x, s->v, s->d, s->tr, s->part, s->m, N, s->eps, s->G, s->bm, dt, n_iter, s->flag, s->stream, bp, s->sym);
        case 5: return launch_dd_step_p<5>(s->x, s->v, s->d, s->tr, s->part, s->m, N, s->eps, s->G, s->bm, dt, n_iter, s->flag, s->stream, bp, s->sym);
        default: set_error("double-double step: unsupported order"); return MH_EINVAL;
    }
}

// nsteps steps: one launched directly, more replayed from a CUDA graph of one
// step (kept while dt and n_iter stay the same).
int dd_advance(mh_dd *sim, double dt, int n_iter, int64_t nsteps)
{
    if (nsteps == 1) return dd_step_once(sim, dt, n_iter);
    if (!sim->graph || sim->graph_dt != dt || sim->graph_n != n_iter) {
        if (sim->graph) { cudaGraphExecDestroy(sim->graph); sim->graph = nullptr; }
        cudaGraph_t g = nullptr;
        MH_CUDA(cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal));
        int rc = dd_step_once(sim, dt, n_iter);
        cudaError_t e = cudaStreamEndCapture(sim->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "double-double step: graph capture");
        e = cudaGraphInstantiate(&sim->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { sim->graph = nullptr; return cuda_fail(e, "double-double step: graph instantiate"); }
        sim->graph_dt = dt;
        sim->graph_n = n_iter;
    }
    for (int64_t k = 0; k < nsteps; ++k) MH_CUDA(cudaGraphLaunch(sim->graph, sim->stream));
    return MH_OK;
}

void dd_count(mh_dd *sim, int n_iter, int64_t nsteps, double pairs_per_eval)
{
    sim->ctr.steps += nsteps;
    sim->ctr.evaluations += nsteps * n_iter;
    sim->ctr.pair_interactions += (double)nsteps * n_iter * pairs_per_eval;
    sim->ctr.particle_steps += (double)nsteps * (double)sim->N;
    const bool reduce = !sim->S && dd_plan((int)sim->N, sim->sym).S > 1;
    sim->ctr.kernel_launches += nsteps * (1 + (reduce ? 3 : 2) * n_iter);
}

int dd_check_flag(mh_dd *s)
{
    if (fault_armed("nonfinite")) {
        set_error("non-finite position or velocity (injected by MH_FAULT=nonfinite)");
        return MH_ENONFINITE;
    }
    int flag = 0;
    MH_CUDA(cudaMemcpyAsync(&flag, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    MH_CUDA(cudaStreamSynchronize(s->stream));
    if (flag) {
        set_error("non-finite position or velocity produced by a double-double step");
        return MH_ENONFINITE;
    }
    return MH_OK;
}

bool finite_all(const double *a, size_t n)
{
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(a[q])) return false;
    return true;
}

// Shared by mh_dd_create and mh_dd_create_batch (offsets, dt: the batch's, or
// null for one system).
int dd_create(mh_dd **out, const char *fn, int64_t N, int order, const double *m, const double *x2,
              const double *v2, double eps, const mh_config *cfg, void *stream, int64_t S,
              const int64_t *offsets, const double *dt)
{
    const std::string f(fn);
    if (order != 4 && order != 6 && order != 8 && order != 10 && order != 12) {
        set_error(f + ": order must be 4, 6, 8, 10 or 12");
        return MH_EINVAL;
    }
    if (!m || !x2 || !v2) { set_error(f + ": m, x2 and v2 are required"); return MH_EINVAL; }
    if (!(eps >= 0.0) || !std::isfinite(eps)) { set_error(f + ": eps must be finite and >= 0"); return MH_EINVAL; }
    mh_config c;
    mh_config_default(&c);
    if (cfg) c = *cfg;
    if (c.beta_mode != MH_BETA_MODIFIED && c.beta_mode != MH_BETA_STANDARD) {
        set_error(f + ": beta_mode must be MH_BETA_MODIFIED or MH_BETA_STANDARD");
        return MH_EINVAL;
    }
    if (!std::isfinite(c.G)) { set_error(f + ": G must be finite"); return MH_EINVAL; }
    if (!finite_all(m, (size_t)N) || !finite_all(x2, (size_t)N * 6) || !finite_all(v2, (size_t)N * 6)) {
        set_error(f + ": non-finite m, x or v");
        return MH_ENONFINITE;
    }
    mh_dd *s = new mh_dd;
    s->N = N;
    s->order = order;
    s->p = order / 2 - 1;
    s->bm = c.beta_mode;
    s->eps = eps;
    s->G = c.G;
    s->S = S;
    const int K = 2 * s->p;
    if (c.symmetric < 0 || c.symmetric > 2) {
        delete s;
        set_error(f + ": symmetric must be 0, 1 or 2");
        return MH_EINVAL;
    }
    s->sym = !S && dd_use_sym((int)N, 6 * s->p, c.symmetric);
    const DDPlan pl = dd_plan((int)N);
    const size_t slots = S ? 1 : std::max((size_t)pl.S, s->sym ? (size_t)dd_plan((int)N, true).S : (size_t)0);
    const size_t R = (size_t)K * 3;      // widest trajectory record (initialisation, P + 1 <= 2p)
    const int nb = (int)((N + kDDThreads - 1) / kDDThreads);
    const size_t ndiag = std::max<size_t>((size_t)nb + 1, (size_t)S);
    auto fail = [&](int rc) { dd_free(s); return rc; };
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
        s->own_stream = true;
    }
    if (fault_armed("alloc")) {
        set_error(f + ": device allocation failed (injected by MH_FAULT=alloc)");
        return fail(MH_ENOMEM);
    }
    bool ok = cudaMalloc((void **)&s->m, N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&s->x, N * 3 * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->v, N * 3 * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->d, N * K * 3 * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->tr, N * R * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->part, slots * N * R * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->diag, ndiag * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void **)&s->flag, sizeof(int)) == cudaSuccess;
    if (ok && S)
        ok = cudaMalloc((void **)&s->off, (S + 1) * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc((void **)&s->sys, N * sizeof(int)) == cudaSuccess &&
             cudaMalloc((void **)&s->dts, S * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error(f + ": device allocation failed");
        return fail(MH_ENOMEM);
    }
    int rc = MH_OK;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (!rc && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), (f + ": upload").c_str());
    };
    std::vector<int> sys_h;
    if (S) {
        sys_h.resize((size_t)N);
        for (int64_t q = 0; q < S; ++q) {
            for (int64_t i = offsets[q]; i < offsets[q + 1]; ++i) sys_h[(size_t)i] = (int)q;
            const double n = (double)(offsets[q + 1] - offsets[q]);
            s->batch_pairs += n * (n - 1.0);
        }
        up(s->off, offsets, (S + 1) * sizeof(int64_t));
        up(s->sys, sys_h.data(), N * sizeof(int));
        up(s->dts, dt, S * sizeof(double));
    }
    up(s->m, m, N * sizeof(double));
    up(s->x, x2, N * 3 * sizeof(double2));
    up(s->v, v2, N * 3 * sizeof(double2));
    if (!rc && cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), (f + ": memset").c_str());
    if (!rc && cudaMemsetAsync(s->d, 0, N * K * 3 * sizeof(double2), s->stream) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), (f + ": memset").c_str());
    if (!rc && s->sym) rc = dd_sym_attrs();
    if (!rc) rc = dd_consts_once(s->stream);
    if (!rc) rc = dd_initialise(s);
    if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), fn);
    if (rc) return fail(rc);
    *out = s;
    return MH_OK;
}

}  // namespace

extern "C" {

int mh_dd_create(mh_dd **out, int64_t N, int order, const double *m, const double *x2, const double *v2,
                 double eps, const mh_config *cfg, void *stream)
{
    if (!out) { set_error("mh_dd_create: out is NULL"); return MH_EINVAL; }
    *out = nullptr;
    if (N < 1 || N > (1 << 24)) { set_error("mh_dd_create: N must be in [1, 2^24]"); return MH_EINVAL; }
    return dd_create(out, "mh_dd_create", N, order, m, x2, v2, eps, cfg, stream, 0, nullptr, nullptr);
}

int mh_dd_create_batch(mh_dd **out, int64_t S, const int64_t *offsets, const double *m, const double *x2,
                       const double *v2, const double *dt, double eps, int order, const mh_config *cfg,
                       void *stream)
{
    if (!out) { set_error("mh_dd_create_batch: out is NULL"); return MH_EINVAL; }
    *out = nullptr;
    if (S < 1 || S > (1 << 22) || !offsets || !dt) {
        set_error("mh_dd_create_batch: need 1 <= S <= 2^22, offsets and dt");
        return MH_EINVAL;
    }
    if (offsets[0] != 0) { set_error("mh_dd_create_batch: offsets[0] must be 0"); return MH_EINVAL; }
    for (int64_t q = 0; q < S; ++q) {
        const int64_t n = offsets[q + 1] - offsets[q];
        if (n < 1 || n > kDDSysMax) {
            set_error("mh_dd_create_batch: every system needs 1 to 64 bodies");
            return MH_EINVAL;
        }
        if (!std::isfinite(dt[q]) || dt[q] == 0.0) {
            set_error("mh_dd_create_batch: every dt must be finite and non-zero");
            return MH_EINVAL;
        }
    }
    const int64_t N = offsets[S];
    if (N > (1 << 24)) { set_error("mh_dd_create_batch: at most 2^24 bodies in all"); return MH_EINVAL; }
    return dd_create(out, "mh_dd_create_batch", N, order, m, x2, v2, eps, cfg, stream, S, offsets, dt);
}

void mh_dd_destroy(mh_dd *sim)
{
    if (sim && sim->stream) cudaStreamSynchronize(sim->stream);
    dd_free(sim);
}

int mh_dd_step(mh_dd *sim, double dt, int n_iter, int64_t nsteps)
{
    if (int rc = dd_check(sim, "mh_dd_step")) return rc;
    if (sim->S) { set_error("mh_dd_step: a batch advances with mh_dd_step_batch"); return MH_EINVAL; }
    if (!std::isfinite(dt) || dt == 0.0) { set_error("mh_dd_step: dt must be finite and non-zero"); return MH_EINVAL; }
    if (n_iter < 1 || n_iter > 64) { set_error("mh_dd_step: n_iter must be in [1, 64]"); return MH_EINVAL; }
    if (nsteps < 0) { set_error("mh_dd_step: nsteps must be >= 0"); return MH_EINVAL; }
    if (int rc = injected_step_fault("mh_dd_step")) return rc;
    NvtxScope range("mh_dd_step");
    if (nsteps == 0) return MH_OK;
    if (int rc = dd_advance(sim, dt, n_iter, nsteps)) return rc;
    for (int64_t k = 0; k < nsteps; ++k) host_add(sim->t_hi, sim->t_lo, dt);
    dd_count(sim, n_iter, nsteps, (double)sim->N * (double)(sim->N - 1));
    return MH_OK;
}

int mh_dd_step_batch(mh_dd *sim, int64_t nsteps, int n_iter)
{
    if (int rc = dd_check(sim, "mh_dd_step_batch")) return rc;
    if (!sim->S) { set_error("mh_dd_step_batch: the handle is not a batch"); return MH_EINVAL; }
    if (n_iter < 1 || n_iter > 64) { set_error("mh_dd_step_batch: n_iter must be in [1, 64]"); return MH_EINVAL; }
    if (nsteps < 0) { set_error("mh_dd_step_batch: nsteps must be >= 0"); return MH_EINVAL; }
    if (int rc = injected_step_fault("mh_dd_step_batch")) return rc;
    NvtxScope range("mh_dd_step_batch");
    if (nsteps == 0) return MH_OK;
    if (int rc = dd_advance(sim, 0.0, n_iter, nsteps)) return rc;     // the steps come from dts
    sim->batch_steps += nsteps;
    dd_count(sim, n_iter, nsteps, sim->batch_pairs);
    return MH_OK;
}

int mh_dd_sync(mh_dd *sim, double *t2, double *x2, double *v2, double *d2)
{
    if (int rc = dd_check(sim, "mh_dd_sync")) return rc;
    const size_t N = (size_t)sim->N, K = 2 * (size_t)sim->p;
    if (x2) MH_CUDA(cudaMemcpyAsync(x2, sim->x, N * 3 * sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
    if (v2) MH_CUDA(cudaMemcpyAsync(v2, sim->v, N * 3 * sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
    if (d2) MH_CUDA(cudaMemcpyAsync(d2, sim->d, N * K * 3 * sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
    if (int rc = dd_check_flag(sim)) return rc;
    if (t2) {
        t2[0] = sim->S ? (double)sim->batch_steps : sim->t_hi;
        t2[1] = sim->S ? 0.0 : sim->t_lo;
    }
    return MH_OK;
}

int mh_dd_set_state(mh_dd *sim, const double *t2, const double *x2, const double *v2, const double *d2)
{
    if (int rc = dd_check(sim, "mh_dd_set_state")) return rc;
    if (!x2 || !v2) { set_error("mh_dd_set_state: x2 and v2 are required"); return MH_EINVAL; }
    const size_t N = (size_t)sim->N, K = 2 * (size_t)sim->p;
    if (!finite_all(x2, N * 6) || !finite_all(v2, N * 6) || (d2 && !finite_all(d2, N * K * 6))) {
        set_error("mh_dd_set_state: non-finite state");
        return MH_ENONFINITE;
    }
    MH_CUDA(cudaMemcpyAsync(sim->x, x2, N * 3 * sizeof(double2), cudaMemcpyHostToDevice, sim->stream));
    MH_CUDA(cudaMemcpyAsync(sim->v, v2, N * 3 * sizeof(double2), cudaMemcpyHostToDevice, sim->stream));
    MH_CUDA(cudaMemsetAsync(sim->flag, 0, sizeof(int), sim->stream));
    if (d2) {
        MH_CUDA(cudaMemcpyAsync(sim->d, d2, N * K * 3 * sizeof(double2), cudaMemcpyHostToDevice, sim->stream));
    } else if (int rc = dd_initialise(sim)) {
        return rc;
    }
    if (t2) {
        if (sim->S) {
            sim->batch_steps = (int64_t)t2[0];
        } else {
            sim->t_hi = t2[0];
            sim->t_lo = t2[1];
        }
    }
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return MH_OK;
}

int mh_dd_diagnostics(mh_dd *sim, double *energy2, double *ecc2, int central)
{
    if (int rc = dd_check(sim, "mh_dd_diagnostics")) return rc;
    if (sim->S) { set_error("mh_dd_diagnostics: a batch reports energies with mh_dd_batch_energy"); return MH_EINVAL; }
    const int N = (int)sim->N;
    if (ecc2 && (central < 0 || central >= N)) { set_error("mh_dd_diagnostics: central out of range"); return MH_EINVAL; }
    const int nb = (N + kDDThreads - 1) / kDDThreads;
    if (energy2) {
        k_dd_energy<<<nb, kDDThreads, 0, sim->stream>>>(sim->m, sim->x, sim->v, N, sim->eps, sim->G, sim->diag);
        MH_LAUNCHED("k_dd_energy");
        k_dd_sum<<<1, 32, 0, sim->stream>>>(sim->diag, nb, sim->diag + nb);
        MH_LAUNCHED("k_dd_sum");
        MH_CUDA(cudaMemcpyAsync(energy2, sim->diag + nb, sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
        sim->ctr.kernel_launches += 2;
    }
    if (ecc2) {
        // the eccentricity vectors are staged in the trajectory buffer (N x 3 fits)
        k_dd_ecc<<<nb, kDDThreads, 0, sim->stream>>>(sim->m, sim->x, sim->v, N, sim->G, central, sim->tr);
        MH_LAUNCHED("k_dd_ecc");
        MH_CUDA(cudaMemcpyAsync(ecc2, sim->tr, (size_t)N * 3 * sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
        sim->ctr.kernel_launches += 1;
    }
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return MH_OK;
}

int mh_dd_batch_energy(mh_dd *sim, double *energy2)
{
    if (int rc = dd_check(sim, "mh_dd_batch_energy")) return rc;
    if (!sim->S) { set_error("mh_dd_batch_energy: the handle is not a batch"); return MH_EINVAL; }
    if (!energy2) { set_error("mh_dd_batch_energy: energy2 is NULL"); return MH_EINVAL; }
    k_dd_energy_sys<<<(unsigned)sim->S, kDDSysMax, 0, sim->stream>>>(sim->m, sim->x, sim->v, sim->off, sim->eps,
                                                                    sim->G, sim->diag);
    MH_LAUNCHED("k_dd_energy_sys");
    sim->ctr.kernel_launches += 1;
    MH_CUDA(cudaMemcpyAsync(energy2, sim->diag, (size_t)sim->S * sizeof(double2), cudaMemcpyDeviceToHost, sim->stream));
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return MH_OK;
}

int mh_dd_pair_eval(int P, int64_t N, const double *m, const double *tr2, double eps, double G, int64_t i0,
                    int64_t i1, int symmetric, double *out2)
{
    const std::string f = "mh_dd_pair_eval";
    if (P < 1 || P > kDDMaxP) { set_error(f + ": P must be 1 .. 5"); return MH_EINVAL; }
    if (N < 1 || N > (int64_t)1 << 24) { set_error(f + ": N must be 1 .. 2^24"); return MH_EINVAL; }
    if (i0 < 0 || i1 > N || i0 > i1) { set_error(f + ": need 0 <= i0 <= i1 <= N"); return MH_EINVAL; }
    if (symmetric < 0 || symmetric > 2) { set_error(f + ": symmetric must be 0, 1 or 2"); return MH_EINVAL; }
    if (!m || !tr2 || (i1 > i0 && !out2)) { set_error(f + ": m, tr2 and out2 are required"); return MH_EINVAL; }
    if (!(eps >= 0.0) || !std::isfinite(eps) || !std::isfinite(G)) { set_error(f + ": eps, G must be finite, eps >= 0"); return MH_EINVAL; }
    if (i1 == i0) return MH_OK;
    const int n = (int)N, R = (P + 1) * 3;
    const bool sym = dd_use_sym(n, R, symmetric);
    const DDPlan pl = dd_plan(n, sym);
    double *dm = nullptr;
    double2 *dtr = nullptr, *dpart = nullptr;
    cudaStream_t st = nullptr;
    int rc = MH_OK;
    auto done = [&](int r) {
        if (st) cudaStreamDestroy(st);
        cudaFree(dm); cudaFree(dtr); cudaFree(dpart);
        return r;
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        st = nullptr;
        return done(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
    }
    if (cudaMalloc((void **)&dm, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&dtr, N * R * sizeof(double2)) != cudaSuccess ||
        cudaMalloc((void **)&dpart, (size_t)pl.S * N * R * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        set_error(f + ": device allocation failed");
        return done(MH_ENOMEM);
    }
    if (sym && (rc = dd_sym_attrs())) return done(rc);
    if ((rc = dd_consts_once(st))) return done(rc);
    if (cudaMemcpyAsync(dm, m, N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dtr, tr2, N * R * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return done(cuda_fail(cudaGetLastError(), "mh_dd_pair_eval: upload"));
    if ((rc = launch_dd_pair(P, dtr, dm, n, eps, G, pl, dpart, st, nullptr))) return done(rc);
    if (pl.S > 1) {
        const int64_t nt = N * R;
        k_dd_add_slots<<<(unsigned)((nt + kDDThreads - 1) / kDDThreads), kDDThreads, 0, st>>>(dpart, pl.S, nt);
        MH_LAUNCHED("k_dd_add_slots");
    }
    if (cudaMemcpyAsync(out2, dpart + (size_t)i0 * R, (size_t)(i1 - i0) * R * sizeof(double2),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return done(cuda_fail(cudaGetLastError(), "mh_dd_pair_eval"));
    return done(MH_OK);
}

int mh_dd_sym_check(int64_t N, int *info)
{
    if (N < 1 || N > (int64_t)1 << 24 || !info) { set_error("mh_dd_sym_check: need 1 <= N <= 2^24 and info"); return MH_EINVAL; }
    const int n = (int)N, nB = (n + kDDSymB - 1) / kDDSymB, items = dd_sym_items(nB), Dmax = nB / 2;
    std::vector<int> pairs((size_t)nB * nB, 0), slots((size_t)nB * nB, 0);   // [I][J], [slot][block]
    for (int t = 0; t < items; ++t) {
        const DDSymItem it = dd_sym_item(t, nB);
        if (it.I < 0 || it.I >= nB || it.b < 0 || it.b > Dmax) { info[2] = t; set_error("mh_dd_sym_check: item out of range"); return MH_EINVAL; }
        const int J = (it.I + it.b) % nB;
        pairs[(size_t)std::min(it.I, J) * nB + std::max(it.I, J)] += 1;
        slots[(size_t)it.b * nB + it.I] += 1;                         // i-side (diagonal: both sides)
        if (it.b > 0) {
            const int sj = ((nB & 1) == 0 && it.b == Dmax) ? it.b : Dmax + it.b;
            if (sj >= nB) { info[2] = t; set_error("mh_dd_sym_check: j-side slot out of range"); return MH_EINVAL; }
            slots[(size_t)sj * nB + J] += 1;
        }
    }
    int bad_pairs = 0, bad_slots = 0;
    for (int I = 0; I < nB; ++I)
        for (int J = I; J < nB; ++J) bad_pairs += pairs[(size_t)I * nB + J] != 1;
    for (size_t q = 0; q < slots.size(); ++q) bad_slots += slots[q] != 1;
    // Inside an item: the kernel's rings (dd_sym_steps, dd_sym_take) take every
    // body pair of two blocks once, and every unordered pair of a block with
    // itself once (no body with itself); no two warps share a subtile in a phase.
    int bad_body_pairs = 0;
    for (int diag = 0; diag < 2; ++diag) {
        std::vector<int> cnt((size_t)kDDSymB * kDDSymB, 0);
        for (int ph = 0; ph < kDDSymW; ++ph) {
            int owner[kDDSymW];
            for (int q = 0; q < kDDSymW; ++q) owner[q] = -1;
            for (int w = 0; w < kDDSymW; ++w) {
                int s0, s1;
                dd_sym_steps(diag != 0, ph, w, s0, s1);
                const int q = (w + ph) % kDDSymW;
                if (s1 > s0) {
                    if (owner[q] >= 0) ++bad_body_pairs;
                    owner[q] = w;
                }
                for (int st = s0; st < s1; ++st)
                    for (int lane = 0; lane < 32; ++lane)
                        if (dd_sym_take(diag != 0, ph, st, lane))
                            ++cnt[(size_t)(32 * w + lane) * kDDSymB + 32 * q + ((lane + st) & 31)];
            }
        }
        for (int a = 0; a < kDDSymB; ++a)
            for (int b = 0; b < kDDSymB; ++b) {
                const int c = cnt[(size_t)a * kDDSymB + b];
                if (!diag) bad_body_pairs += c != 1;
                else if (a == b) bad_body_pairs += c != 0;
                else if (a < b) bad_body_pairs += c + cnt[(size_t)b * kDDSymB + a] != 1;
            }
    }
    info[0] = nB;
    info[1] = items;
    info[2] = bad_pairs;
    info[3] = bad_slots;
    info[4] = bad_body_pairs;
    if (bad_pairs || bad_slots || bad_body_pairs) {
        set_error("mh_dd_sym_check: block pairs, body pairs or slots not covered exactly once");
        return MH_EINVAL;
    }
    return MH_OK;
}

int mh_dd_info(mh_dd *sim, int64_t *N, int *order, mh_counters *counters)
{
    if (int rc = dd_check(sim, "mh_dd_info")) return rc;
    if (N) *N = sim->N;
    if (order) *order = sim->order;
    if (counters) *counters = sim->ctr;
    return MH_OK;
}

}  // extern "C"
