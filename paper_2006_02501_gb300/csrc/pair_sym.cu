// FP64 all-pairs evaluation of a^(0..P) that computes every unordered pair once
// (the E of P(EC)^n under shared steps, and the initialisation passes P <= 5).
//
// Pair physics (Dittmann 2020, Section 3, intro): a_ij = G m_j r_ij s^(-3/2).
// With the scaled terms B_k of pair_math.cuh, body i receives G m_j S B_k(i,j)
// and body j receives G m_i S B_k(j,i) = -G m_i S B_k(i,j): the terms are odd
// under i <-> j and S, alpha, beta, gamma are even.  One evaluation of the pair
// therefore serves both bodies, and an interaction costs about 96 FP64
// operations per unordered pair instead of 2 x 83 for two ordered pairs.  On a
// part with two FP64 lanes per SM this halves the time of the FP64 form; the
// extra data movement (shuffles, shared memory) runs on otherwise idle pipes.
//
// Decomposition.  Bodies are cut into blocks of R = 128 (the padded count Np is
// a multiple of R; nB blocks).  Block row I handles the diagonal block (I, I)
// and the blocks J = I + b (mod nB), b = 1 .. D with D = floor(nB/2); when nB
// is even (always, for the simulation's padding to 256) the block pair at
// b = nB/2 is done by the rows I < nB/2 only.  Every unordered block pair is
// then done exactly once and every row has the same amount of work, to one
// block.  A row is cut into C chunks of Bc consecutive distances; an item is
// one (row, chunk).  An item runs its distances from the largest down, the
// diagonal block last.
//
// Inside a CTA (4 warps) warp w holds the 32 i-bodies I*R + 32w + lane.  For
// an off-diagonal block the warps take the block's four 32-body j-subtiles in
// a rotation (warp w takes subtile (w + jt) mod 4 at stage jt); a warp runs the
// 32 x 32 pairs of a subtile as a ring: each lane holds one j-body with its
// j-side accumulator and passes both one lane on after every pair.  The j-side
// sums of a subtile move between warps through shared memory at the stage
// barriers.  The diagonal block is evaluated as ordered pairs (i-side only,
// the i == j pair guarded).
//
// Output: C (1 + G) partial-sum slots, O(N C) memory.  Slot ch < C holds the
// i-side sums of row chunk ch (registers over the whole item, one plain store).
// The j-side sums that the rows' chunk ch add into block J go to one of G
// chains by row mod G; chain g of (ch, J) is one slot, into which its rows add
// one after another in a fixed order (a serial reduction): a counter per
// (chunk, chain, block) says how many have done so, and a row waits until the
// counter equals its rank.  The order is, for a launch whose items all run at
// once (one item per CTA), descending distance; otherwise ascending row index,
// with items handed out in that order by an atomic counter.  In both orders the
// writer before row I in its chain is usually row I - G at distance b + G,
// which the descending-distance sweep reaches G blocks earlier: rows that run
// at somewhat different speeds (CTAs share their SM with different neighbours)
// still rarely wait.  The corrector adds the slots in a fixed order: results
// are deterministic and independent of which CTA ran which item.
//
// Every wait is bounded in time.  A wait that runs out sets a bit in the
// simulation's status word and the CTA goes on (its sums are then invalid and
// the host reports MH_ETIMEOUT); later waits of the launch see the bit and do
// not wait.  No CTA waits on an item that has not been handed out: in the
// ascending-row order every writer before row I has a smaller row index and
// was handed out earlier, and a one-item-per-CTA launch is planned only when
// all its CTAs are resident at once.
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

constexpr int kSymWarps = 4;
constexpr int kSymR = 32 * kSymWarps;     // bodies per block
// Accumulation chains per j-slot: the writer before row I in its chain is row
// I - G, which reaches the block G sweeps earlier, so a row may run up to G - 1
// blocks ahead of the rows before it without waiting.
constexpr int kSymChains = 4;

// Schedule of one launch (from SymPlan) and the ordered-accumulation words.
struct SymSched {
    int nB, D, C, Bc;
    int G;                 // accumulation chains per j-slot: writer rows are split by row mod G
    int cyclic;            // 1: one item per CTA, all resident; writers by descending distance
    int items;             // nB * C
    unsigned *fetch;       // [1] next item to hand out (multi-wave order); reset by the launch's last fetch
    unsigned *count;       // [C][G][nB] writes done into j-slot (ch, g, J) in this launch; 0 between launches
    int *flag;             // status word: kFlagSymWait when a wait ran out
    unsigned long long wait_ns;   // limit of one wait
    unsigned bias;         // added to every awaited count (0 unless a host-injected fault asks otherwise)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0: the CTA's next item (>= items once there is none).  The fetches of
// a launch number items + gridDim.x; the last one resets the counter.
__device__ __forceinline__ unsigned next_item(const SymSched &sc, int n)
{
    if (sc.cyclic) return n == 0 ? blockIdx.x : 0xffffffffu;
    const unsigned v = atomicAdd(sc.fetch, 1u);
    if (v == (unsigned)sc.items + gridDim.x - 1u) atomicExch(sc.fetch, 0u);
    return v;
}

// The rows that add into j-slot (ch, g, J): I' = J - b (mod nB) for the
// distances b >= 1 of chunk ch that row I' evaluates, with I' = g (mod G).
// Returns how many there are and, in *rank, how many of them come before row I
// (which evaluates J at distance bI).
__host__ __device__ __forceinline__ int j_writers(const SymSched &sc, int J, int ch, int g, int I, int bI,
                                                  int *rank)
{
    const bool even = (sc.nB & 1) == 0;
    const int lo = ch * sc.Bc > 1 ? ch * sc.Bc : 1;
    const int hi = ch * sc.Bc + sc.Bc < sc.D + 1 ? ch * sc.Bc + sc.Bc : sc.D + 1;
    int nw = 0, rk = 0;
    for (int b = lo; b < hi; ++b) {
        int r = J - b;
        if (r < 0) r += sc.nB;
        if (even && b == sc.D && r >= sc.nB / 2) continue;   // rows >= nB/2 skip distance nB/2
        if (r % sc.G != g) continue;
        ++nw;
        rk += sc.cyclic ? (b > bI) : (r < I);
    }
    *rank = rk;
    return nw;
}

// Thread 0: wait, bounded in time, until *c == want.
__device__ __noinline__ void wait_turn(const unsigned *c, unsigned want, const SymSched &sc)
{
    if (ld_acquire(c) == want) return;
    const unsigned long long t0 = now_ns();
    for (int it = 0;; ++it) {
        __nanosleep(it < 32 ? 20 : 200);
        if (ld_acquire(c) == want) return;
        if ((*(volatile int *)sc.flag & kFlagSymWait) || now_ns() - t0 > sc.wait_ns) {
            atomicOr(sc.flag, kFlagSymWait);
            return;
        }
    }
}

// Shared-memory words of one CTA for the ordered flush.
struct FlushSmem {
    int item, rank, next;
    unsigned zero;        // bit g: j-slot (ch, g) of the item's own block has no writer
};

// Thread 0 at the start of item (I, ch): which of block I's j-slots of chunk ch
// no row adds into (they must hold zeros).
__device__ __forceinline__ unsigned unwritten_chains(const SymSched &sc, int I, int ch)
{
    unsigned z = 0;
    for (int g = 0; g < sc.G; ++g) {
        int rk;
        if (j_writers(sc, I, ch, g, I, 0, &rk) == 0) z |= 1u << g;
    }
    return z;
}

// j-slot of chunk ch, chain g (the i-side slots come first).
__host__ __device__ __forceinline__ int64_t j_slot(const SymSched &sc, int ch, int g)
{
    return (int64_t)sc.C + (int64_t)ch * sc.G + g;
}

// Thread 0 before row I's ordered flush into j-slot (ch, I mod G, J): wait for
// its turn and publish the rank (0: this row writes first) to the CTA.
__device__ __forceinline__ void flush_begin(const SymSched &sc, FlushSmem &fs, int I, int J, int ch, int b)
{
    if (threadIdx.x == 0) {
        const int g = I % sc.G;
        int rank = 0;
        const int nw = j_writers(sc, J, ch, g, I, b, &rank);
        fs.rank = rank;
        fs.next = rank + 1 == nw ? 0 : rank + 1;
        if (rank > 0) wait_turn(&sc.count[(j_slot(sc, ch, g) - sc.C) * sc.nB + J], (unsigned)rank + sc.bias, sc);
    }
}

// Thread 0 after the CTA's stores of the flush (behind a barrier): pass the
// turn on with a release store, which orders the whole CTA's stores before it
// (the last writer leaves the counter at 0).
__device__ __forceinline__ void flush_end(const SymSched &sc, const FlushSmem &fs, int I, int J, int ch)
{
    if (threadIdx.x == 0)
        st_release(&sc.count[(j_slot(sc, ch, I % sc.G) - sc.C) * sc.nB + J], (unsigned)fs.next);
}

template <int P>
struct SymArgs {
    const double *jrec;   // [3(P+1)][ld]
    const double *m;      // [ld]
    int64_t ld;           // row stride (the padded body count, a multiple of kSymR)
    int64_t N;            // bodies; positions N .. ld-1 are padding
    SymSched sc;
    double eps2, G;
    double *part;         // [2C][(P+1)*3][ld]
    unsigned long long *wmax;   // kH: max over pairs of G (m_i + m_j) s^(-3/2) (bit pattern), raised
};

// Record of body b.  Padding bodies get mass 0 and distinct far-away positions,
// so that no pair has r = 0 (their own sums are never read).
template <int P>
__device__ __forceinline__ void load_body(const SymArgs<P> &a, int64_t b, double (&r)[P + 1][3], double &gm)
{
    if (b < a.N) {
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = a.jrec[(3 * k + c) * a.ld + b];
        gm = a.G * a.m[b];
    } else {
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = 0.0;
        r[0][0] = kFarAway + (double)(b - a.N);
        gm = 0.0;
    }
}

template <int P>
__device__ __forceinline__ void rotate(double (&r)[P + 1][3], double &gm, int src)
{
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) r[k][c] = __shfl_sync(0xffffffffu, r[k][c], src);
    gm = __shfl_sync(0xffffffffu, gm, src);
}

// kH: also track w = G (m_i + m_j) s^(-3/2) over all pairs i != j, whose maximum
// gives the time-step criterion of Section 3.3 (Eq. 24: H = eta w_max^(-1/2)).
// Non-negative doubles order as their bit patterns, so the maximum is an
// integer maximum (off the FP64 pipe) and the result does not depend on the
// order of the pairs.
template <int P, bool kH>
__global__ void __launch_bounds__(kSymR, P <= 3 ? 3 : 2) k_pair_fp64_sym(SymArgs<P> a)
{
    constexpr int NR = 3 * (P + 1);
    const SymSched &sc = a.sc;
    unsigned long long wm = 0ull;
    __shared__ double accs[NR][kSymR];    // j-side sums of the current block, by column
    __shared__ FlushSmem fs;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;      // ring: after t passes lane l holds j-lane (l + t) mod 32
    const bool even = (sc.nB & 1) == 0;
    for (int n = 0;; ++n) {
        if (threadIdx.x == 0) fs.item = (int)min(next_item(sc, n), (unsigned)sc.items);
        __syncthreads();
        const int item = fs.item;
        if (item >= sc.items) break;
        const int I = item / sc.C;
        const int ch = item % sc.C;
        if (threadIdx.x == 0) fs.zero = unwritten_chains(sc, I, ch);
        const int64_t ib = (int64_t)I * kSymR + threadIdx.x;
        double ri[P + 1][3], gmi;
        load_body<P>(a, ib, ri, gmi);
        double acci[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acci[k][c] = 0.0;
        __syncthreads();
        for (int g = 0; g < sc.G; ++g)
            if (fs.zero >> g & 1u) {
                // no row adds into this j-slot of the block: it holds zeros
                double *out = a.part + j_slot(sc, ch, g) * NR * a.ld + ib;
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
            }

        const int dmax = (even && I >= sc.nB / 2) ? sc.D - 1 : sc.D;
        const int b0 = ch * sc.Bc;
        const int b1 = min(b0 + sc.Bc, dmax + 1);
        for (int b = b1 - 1; b >= b0; --b) {
            if (b == 0) {
                // diagonal block: ordered pairs into the i-side only
                for (int js = 0; js < kSymWarps; ++js) {
                    double rj[P + 1][3], gmj;
                    load_body<P>(a, (int64_t)I * kSymR + js * 32 + lane, rj, gmj);
                    for (int t = 0; t < 32; ++t) {
                        const bool self = js == w && t == 0;
                        double r[P + 1][3];
#pragma unroll
                        for (int k = 0; k <= P; ++k)
#pragma unroll
                            for (int c = 0; c < 3; ++c) r[k][c] = rj[k][c] - ri[k][c];
                        double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
                        s = self ? 1.0 : s;
                        const double wi = self ? 0.0 : gmj;
                        const double rinv = rsqrt_fp64(s);
                        const double sinv = rinv * rinv;
                        const double S = rinv * sinv;
                        const double mS = wi * S;
                        if constexpr (kH) {
                            const unsigned long long wb = self ? 0ull : (unsigned long long)__double_as_longlong((gmi + gmj) * S);
                            wm = wb > wm ? wb : wm;
                        }
                        pair_odd_terms<P, double>(r, sinv, [&](int k, int c, double B) {
                            acci[k][c] = fma(mS, B, acci[k][c]);
                        });
                        rotate<P>(rj, gmj, src);
                    }
                }
                continue;
            }
            const int J = (I + b) % sc.nB;
            for (int jt = 0; jt < kSymWarps; ++jt) {
                const int js = (w + jt) % kSymWarps;
                double rj[P + 1][3], gmj, accj[P + 1][3];
                load_body<P>(a, (int64_t)J * kSymR + js * 32 + lane, rj, gmj);
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accj[k][c] = jt == 0 ? 0.0 : accs[3 * k + c][js * 32 + lane];
                for (int t = 0; t < 32; ++t) {
                    double r[P + 1][3];
#pragma unroll
                    for (int k = 0; k <= P; ++k)
#pragma unroll
                        for (int c = 0; c < 3; ++c) r[k][c] = rj[k][c] - ri[k][c];
                    const double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
                    const double rinv = rsqrt_fp64(s);
                    const double sinv = rinv * rinv;
                    const double S = rinv * sinv;
                    const double wi = gmj * S, wj = gmi * S;
                    if constexpr (kH) {
                        const unsigned long long wb = (unsigned long long)__double_as_longlong(wi + wj);
                        wm = wb > wm ? wb : wm;
                    }
                    pair_odd_terms<P, double>(r, sinv, [&](int k, int c, double B) {
                        acci[k][c] = fma(wi, B, acci[k][c]);
                        accj[k][c] = fma(-wj, B, accj[k][c]);
                    });
                    rotate<P>(rj, gmj, src);
#pragma unroll
                    for (int k = 0; k <= P; ++k)
#pragma unroll
                        for (int c = 0; c < 3; ++c) accj[k][c] = __shfl_sync(0xffffffffu, accj[k][c], src);
                }
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accs[3 * k + c][js * 32 + lane] = accj[k][c];
                __syncthreads();
            }
            // ordered flush of block J's j-side sums into j-slot (ch, J)
            flush_begin(sc, fs, I, J, ch, b);
            __syncthreads();
            const bool add = fs.rank > 0;
            double *out = a.part + j_slot(sc, ch, I % sc.G) * NR * a.ld + (int64_t)J * kSymR + threadIdx.x;
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const double v = accs[q][threadIdx.x];
                __stcg(out + q * a.ld, add ? __ldcg(out + q * a.ld) + v : v);
            }
            __syncthreads();
            flush_end(sc, fs, I, J, ch);
        }
        double *out = a.part + (int64_t)ch * NR * a.ld + ib;
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) out[(3 * k + c) * a.ld] = acci[k][c];
    }
    if constexpr (kH) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xffffffffu, wm, o);
            wm = q > wm ? q : wm;
        }
        if (lane == 0 && wm) atomicMax(a.wmax, wm);
    }
}

// Launch configuration: a plan with one item per CTA is launched cooperatively,
// so that the runtime makes all its CTAs resident at once (its turns wait on
// CTAs of the same launch in any order); otherwise a plain launch.
struct SymLaunch {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    SymLaunch(const SymPlan &pl, int threads, cudaStream_t st)
    {
        cfg.gridDim = dim3((unsigned)pl.grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = pl.cyclic ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
};

SymSched make_sched(const SymPlan &pl, const SymSync &sy)
{
    return SymSched{pl.nB, pl.D, pl.C, pl.Bc, pl.G, pl.cyclic ? 1 : 0, pl.nB * pl.C, sy.words, sy.words + 1,
                    sy.flag, sy.wait_ns, sy.bias};
}

template <int P>
int launch_sym(const SymPlan &pl, const SymSync &sy, const double *jrec, const double *m, int64_t ld, int64_t N,
               double eps, double G, double *part, unsigned long long *wmax, cudaStream_t st)
{
    SymArgs<P> a{jrec, m, ld, N, make_sched(pl, sy), eps * eps, G, part, wmax};
    const SymLaunch l(pl, kSymR, st);
    if (wmax)
        MH_CUDA(cudaLaunchKernelEx(&l.cfg, k_pair_fp64_sym<P, true>, a));
    else
        MH_CUDA(cudaLaunchKernelEx(&l.cfg, k_pair_fp64_sym<P, false>, a));
    return MH_OK;
}

// ---------------------------------------------------------------------------
// FP32-pair form, each unordered pair once.  Same block schedule, ring and
// ordered j-side accumulation as the FP64 kernel above; the pair arithmetic is
// the precision form's: x and v differences from the hi/lo split,
// (hi_j - hi_i) + (lo_j - lo_i), everything else of the pair in FP32.
// ---------------------------------------------------------------------------

template <int P>
struct SymArgs32 {
    const float *jrec32;  // [nf32(P)][ld]: x_hi, x_lo, v_hi, v_lo, a, a-dot, G m
    int64_t ld, N;
    SymSched sc;
    float eps2;
    double *part;         // [2C][(P+1)*3][ld]
};

template <int P>
struct Rec32s {
    static constexpr int NF = nf32(P);
};

// Record of body b; padding bodies massless at distinct far-away positions.
template <int P>
__device__ __forceinline__ void load_body32(const SymArgs32<P> &a, int64_t b, float (&r)[Rec32s<P>::NF])
{
    constexpr int NF = Rec32s<P>::NF;
    if (b < a.N) {
#pragma unroll
        for (int q = 0; q < NF; ++q) r[q] = a.jrec32[q * a.ld + b];
    } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) r[q] = 0.0f;
        r[0] = (float)kFarAway + (float)(b - a.N);
    }
}

// Two warps per CTA, two i-bodies per lane: lane l of warp w holds the bodies
// of i-subtiles 2w and 2w + 1 in the two lanes of Blackwell's paired FP32
// instructions (FFMA2/FMUL2/FADD2), so every j-record passed around the ring
// serves two pairs and one issue slot advances both.  The i-side sums are
// packed too; the j-side sum of a ring lane adds both pairs' terms in FP32.
// FP32 sums cover one 128-body block (as the tiles of the ordered kernels) and
// are added to FP64 once per block.
constexpr int kSym32Warps = 2;

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// The scaled terms B_k of pair_abg_terms for two pairs at once (negated
// coefficients so that every update is one multiply-add); sink(k, c, B).
template <int P, typename Sink>
__device__ __forceinline__ void pair_abg_terms_x2(const float2 (&r)[P + 1][3], float2 sinv, Sink &&sink)
{
    const float2 rv = fma2(r[0][2], r[1][2], fma2(r[0][1], r[1][1], mul2(r[0][0], r[1][0])));
    const float2 al = mul2(rv, sinv);
    const float2 na3 = mul2(f2(-3.0f), al);
    float2 B1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B1[c] = fma2(na3, r[0][c], r[1][c]);
        sink(0, c, r[0][c]);
        sink(1, c, B1[c]);
    }
    if constexpr (P >= 2) {
        const float2 al2 = mul2(al, al);
        float2 w2 = mul2(r[1][0], r[1][0]);
        w2 = fma2(r[1][1], r[1][1], w2);
        w2 = fma2(r[1][2], r[1][2], w2);
        w2 = fma2(r[0][0], r[2][0], w2);
        w2 = fma2(r[0][1], r[2][1], w2);
        w2 = fma2(r[0][2], r[2][2], w2);
        const float2 be = fma2(w2, sinv, al2);
        const float2 na6 = mul2(f2(-6.0f), al), nb3 = mul2(f2(-3.0f), be);
        float2 B2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B2[c] = fma2(nb3, r[0][c], fma2(na6, B1[c], r[2][c]));
            sink(2, c, B2[c]);
        }
        if constexpr (P >= 3) {
            const float2 va = fma2(r[1][2], r[2][2], fma2(r[1][1], r[2][1], mul2(r[1][0], r[2][0])));
            const float2 rj = fma2(r[0][2], r[3][2], fma2(r[0][1], r[3][1], mul2(r[0][0], r[3][0])));
            const float2 w3 = fma2(f2(3.0f), va, rj);
            // gamma = w3/s + alpha (3 beta - 4 alpha^2), 3 beta - 4 alpha^2 = -(nb3 + 4 alpha^2)
            const float2 u = fma2(f2(4.0f), al2, nb3);
            const float2 ga = fma2(w3, sinv, mul2(mul2(f2(-1.0f), al), u));
            const float2 na9 = mul2(f2(-9.0f), al), nb9 = mul2(f2(-9.0f), be), ng3 = mul2(f2(-3.0f), ga);
#pragma unroll
            for (int c = 0; c < 3; ++c) sink(3, c, fma2(ng3, r[0][c], fma2(nb9, B1[c], fma2(na9, B2[c], r[3][c]))));
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32 * kSym32Warps, 4) k_pair_fp32_sym(SymArgs32<P> a)
{
    constexpr int NF = Rec32s<P>::NF;
    constexpr int NR = 3 * (P + 1);
    const SymSched &sc = a.sc;
    __shared__ float accs[NR][kSymR];     // j-side FP32 sums of the current block, by column
    __shared__ FlushSmem fs;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;
    const bool even = (sc.nB & 1) == 0;
    const float2 eps2 = f2(a.eps2);
    for (int n = 0;; ++n) {
        if (threadIdx.x == 0) fs.item = (int)min(next_item(sc, n), (unsigned)sc.items);
        __syncthreads();
        const int item = fs.item;
        if (item >= sc.items) break;
        const int I = item / sc.C;
        const int ch = item % sc.C;
        if (threadIdx.x == 0) fs.zero = unwritten_chains(sc, I, ch);
        // the lane's two i-bodies, negated (differences become additions), packed
        float2 ni[NF - 1], gmi;
        {
            float r0[NF], r1[NF];
            load_body32<P>(a, (int64_t)I * kSymR + (2 * w) * 32 + lane, r0);
            load_body32<P>(a, (int64_t)I * kSymR + (2 * w + 1) * 32 + lane, r1);
#pragma unroll
            for (int q = 0; q < NF - 1; ++q) ni[q] = make_float2(-r0[q], -r1[q]);
            gmi = make_float2(r0[NF - 1], r1[NF - 1]);
        }
        double acc64[2][NR];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc64[k][q] = 0.0;
        __syncthreads();
        for (int g = 0; g < sc.G; ++g)
            if (fs.zero >> g & 1u) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    double *out = a.part + j_slot(sc, ch, g) * NR * a.ld + (int64_t)I * kSymR + threadIdx.x + k * 64;
#pragma unroll
                    for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
                }
            }

        const int dmax = (even && I >= sc.nB / 2) ? sc.D - 1 : sc.D;
        const int b0 = ch * sc.Bc;
        const int b1 = min(b0 + sc.Bc, dmax + 1);
        for (int b = b1 - 1; b >= b0; --b) {
            const bool diag = b == 0;
            const int J = (I + b) % sc.nB;
            float2 acci[P + 1][3];
#pragma unroll
            for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                for (int c = 0; c < 3; ++c) acci[n2][c] = f2(0.0f);
            for (int jt = 0; jt < 4; ++jt) {
                // off-diagonal: at stage jt warp w takes j-subtile (2w + jt) mod 4 (the two
                // warps never share one); diagonal block: every warp takes every subtile
                const int js = diag ? jt : (2 * w + jt) & 3;
                float rj[NF];
                load_body32<P>(a, (int64_t)J * kSymR + js * 32 + lane, rj);
                float accj[P + 1][3];
#pragma unroll
                for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accj[n2][c] = 0.0f;
                for (int t = 0; t < 32; ++t) {
                    float2 r[P + 1][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        r[0][c] = add2(add2(f2(rj[c]), ni[c]), add2(f2(rj[3 + c]), ni[3 + c]));
                        r[1][c] = add2(add2(f2(rj[6 + c]), ni[6 + c]), add2(f2(rj[9 + c]), ni[9 + c]));
                        if constexpr (P >= 2) r[2][c] = add2(f2(rj[12 + c]), ni[12 + c]);
                        if constexpr (P >= 3) r[3][c] = add2(f2(rj[15 + c]), ni[15 + c]);
                    }
                    float2 s = fma2(r[0][0], r[0][0], fma2(r[0][1], r[0][1], fma2(r[0][2], r[0][2], eps2)));
                    const bool self0 = diag && js == 2 * w && t == 0;
                    const bool self1 = diag && js == 2 * w + 1 && t == 0;
                    s.x = self0 ? 1.0f : s.x;
                    s.y = self1 ? 1.0f : s.y;
                    const float2 rinv = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
                    const float2 sinv = mul2(rinv, rinv);
                    const float2 S = mul2(rinv, sinv);
                    float2 wi = mul2(f2(rj[NF - 1]), S);
                    wi.x = self0 ? 0.0f : wi.x;
                    wi.y = self1 ? 0.0f : wi.y;
                    const float2 wj = diag ? f2(0.0f) : mul2(gmi, S);
                    pair_abg_terms_x2<P>(r, sinv, [&](int n3, int c, float2 B) {
                        acci[n3][c] = fma2(wi, B, acci[n3][c]);
                        accj[n3][c] = fmaf(-wj.y, B.y, fmaf(-wj.x, B.x, accj[n3][c]));
                    });
#pragma unroll
                    for (int q = 0; q < NF; ++q) rj[q] = __shfl_sync(0xffffffffu, rj[q], src);
                    if (!diag) {
#pragma unroll
                        for (int n3 = 0; n3 <= P; ++n3)
#pragma unroll
                            for (int c = 0; c < 3; ++c) accj[n3][c] = __shfl_sync(0xffffffffu, accj[n3][c], src);
                    }
                }
                if (!diag) {
                    // each column is visited twice, by warp 0 and by warp 1: first at stage
                    // 0 (columns 0, 2) or 1 (columns 1, 3), second at stage 2 or 3
#pragma unroll
                    for (int n3 = 0; n3 <= P; ++n3)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float &cell = accs[3 * n3 + c][js * 32 + lane];
                            cell = (jt < 2 ? 0.0f : cell) + accj[n3][c];
                        }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc64[0][3 * n2 + c] += (double)acci[n2][c].x;
                    acc64[1][3 * n2 + c] += (double)acci[n2][c].y;
                }
            if (!diag) {
                // ordered flush of block J's j-side sums into j-slot (ch, J)
                flush_begin(sc, fs, I, J, ch, b);
                __syncthreads();
                const bool add = fs.rank > 0;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int col = threadIdx.x + k * 64;
                    double *out = a.part + j_slot(sc, ch, I % sc.G) * NR * a.ld + (int64_t)J * kSymR + col;
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        const double v = (double)accs[q][col];
                        __stcg(out + q * a.ld, add ? __ldcg(out + q * a.ld) + v : v);
                    }
                }
                __syncthreads();
                flush_end(sc, fs, I, J, ch);
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            double *out = a.part + (int64_t)ch * NR * a.ld + (int64_t)I * kSymR + (2 * w + k) * 32 + lane;
#pragma unroll
            for (int q = 0; q < NR; ++q) out[q * a.ld] = acc64[k][q];
        }
    }
}

template <int P>
int launch_sym32(const SymPlan &pl, const SymSync &sy, const float *jrec32, int64_t ld, int64_t N, double eps,
                 double *part, cudaStream_t st)
{
    SymArgs32<P> a{jrec32, ld, N, make_sched(pl, sy), (float)(eps * eps), part};
    const SymLaunch l(pl, 32 * kSym32Warps, st);
    MH_CUDA(cudaLaunchKernelEx(&l.cfg, k_pair_fp32_sym<P>, a));
    return MH_OK;
}

}  // namespace

// The plan for `slots` resident CTAs (items of equal size; the chunk count with
// the fewest block-times on the busiest CTA).  One item per CTA when they all fit
// at once (distance order); otherwise the CTAs take items in row order, and rows
// at the end of a launch that is only just above one wave wait for the first
// rows (their blocks near the wrap-around come last in that order): count one
// wave more.
SymPlan plan_sym_slots(int64_t ld, int slots)
{
    SymPlan pl{};
    if (ld % kSymR != 0 || ld < kSymR || slots < 1) return pl;
    pl.nB = (int)(ld / kSymR);
    pl.D = pl.nB / 2;
    const int nb = pl.D + 1;                        // blocks of the longest row
    double best = 1e300;
    for (int C = 1; C <= nb; ++C) {
        const int Bc = (nb + C - 1) / C;
        if ((nb + Bc - 1) / Bc != C) continue;
        const int64_t items = (int64_t)pl.nB * C;
        const bool cyclic = items <= slots;
        int64_t waves = cyclic ? 1 : (items + slots - 1) / slots;
        if (!cyclic && items < slots + nb) waves += 1;
        const double cost = (double)waves * (Bc + 1.0) * (1.0 + 0.001 * C);
        if (cost < best) {
            best = cost;
            pl.C = C;
            pl.Bc = Bc;
            pl.cyclic = cyclic;
        }
    }
    const int64_t items = (int64_t)pl.nB * pl.C;
    pl.grid = (int)(pl.cyclic ? items : std::min<int64_t>(items, slots));
    pl.G = std::min(kSymChains, std::max(pl.Bc - 1, 1));
    pl.slots = pl.C * (1 + pl.G);
    pl.sync_words = 1 + pl.C * pl.G * pl.nB;
    return pl;
}

SymPlan plan_sym(int P, int64_t ld, int device, bool fp32)
{
    if (ld % kSymR != 0 || ld < kSymR || P < 1 || P > (fp32 ? 3 : 5)) return SymPlan{};
    // resident CTAs per device, cached per (device, P, form)
    static int slot_cache[64][16] = {{0}};
    const int ci = P + (fp32 ? 8 : 0);
    int slots = device >= 0 && device < 64 ? slot_cache[device][ci] : 0;
    if (slots == 0) {
        int n_sm = 0, occ = 0;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (fp32) {
            const void *fn = P == 1 ? (const void *)k_pair_fp32_sym<1>
                           : P == 2 ? (const void *)k_pair_fp32_sym<2> : (const void *)k_pair_fp32_sym<3>;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * kSym32Warps, 0);
        } else {
            const void *fn = P == 1 ? (const void *)k_pair_fp64_sym<1, false>
                           : P == 2 ? (const void *)k_pair_fp64_sym<2, false>
                           : P == 3 ? (const void *)k_pair_fp64_sym<3, false>
                           : P == 4 ? (const void *)k_pair_fp64_sym<4, false> : (const void *)k_pair_fp64_sym<5, false>;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSymR, 0);
        }
        slots = std::max(n_sm, 1) * std::max(occ, 1);
        if (device >= 0 && device < 64) slot_cache[device][ci] = slots;
    }
    return plan_sym_slots(ld, slots);
}

int launch_pair_sym32(int P, const SymPlan &pl, const SymSync &sy, const float *jrec32, int64_t ld, int64_t N,
                      double eps, double *part, cudaStream_t st)
{
    switch (P) {
    case 1: return launch_sym32<1>(pl, sy, jrec32, ld, N, eps, part, st);
    case 2: return launch_sym32<2>(pl, sy, jrec32, ld, N, eps, part, st);
    case 3: return launch_sym32<3>(pl, sy, jrec32, ld, N, eps, part, st);
    }
    set_error("launch_pair_sym32: P must be 1..3");
    return MH_EINVAL;
}

int launch_pair_sym(int P, const SymPlan &pl, const SymSync &sy, const double *jrec, const double *m, int64_t ld,
                    int64_t N, double eps, double G, double *part, cudaStream_t st, unsigned long long *wmax)
{
    switch (P) {
    case 1: return launch_sym<1>(pl, sy, jrec, m, ld, N, eps, G, part, wmax, st);
    case 2: return launch_sym<2>(pl, sy, jrec, m, ld, N, eps, G, part, wmax, st);
    case 3: return launch_sym<3>(pl, sy, jrec, m, ld, N, eps, G, part, wmax, st);
    case 4: return launch_sym<4>(pl, sy, jrec, m, ld, N, eps, G, part, wmax, st);
    case 5: return launch_sym<5>(pl, sy, jrec, m, ld, N, eps, G, part, wmax, st);
    }
    set_error("launch_pair_sym: P must be 1..5");
    return MH_EINVAL;
}

// Host check of the ordered accumulation of a plan (used by the CPU tests):
// every j-slot's writers hold the ranks 0 .. nw-1 once each, slots without
// writers are the ones that are zeroed, and every wait is on a writer that
// cannot be waiting on it in turn: in the row order one handed out earlier, in
// the distance order one at a larger distance (so the waits of a launch whose
// CTAs are all resident form no cycle).
int sym_schedule_check(int64_t ld, int slots, int *info)
{
    const SymPlan pl = plan_sym_slots(ld, slots);
    if (pl.nB == 0) return MH_EINVAL;
    SymSched sc{pl.nB, pl.D, pl.C, pl.Bc, pl.G, pl.cyclic ? 1 : 0, pl.nB * pl.C, nullptr, nullptr, nullptr, 0, 0};
    const bool even = (pl.nB & 1) == 0;
    const int64_t nslot = (int64_t)pl.C * pl.G * pl.nB;
    std::vector<int> seen(nslot, 0), nwv(nslot, -1);
    std::vector<std::vector<std::pair<int, int>>> by_rank(nslot);   // rank -> (item, distance)
    for (int item = 0; item < sc.items; ++item) {
        const int I = item / sc.C, ch = item % sc.C;
        const int dmax = (even && I >= sc.nB / 2) ? sc.D - 1 : sc.D;
        const int b0 = ch * sc.Bc, b1 = std::min(b0 + sc.Bc, dmax + 1);
        for (int b = b1 - 1; b >= b0 && b >= 1; --b) {
            const int J = (I + b) % sc.nB;
            const int g = I % sc.G;
            int rank = 0;
            const int nw = j_writers(sc, J, ch, g, I, b, &rank);
            const int64_t q = (j_slot(sc, ch, g) - sc.C) * sc.nB + J;
            if (nwv[q] < 0) {
                nwv[q] = nw;
                by_rank[q].assign(nw, {-1, -1});
            }
            if (nwv[q] != nw || rank < 0 || rank >= nw || by_rank[q][rank].first >= 0) return 1;
            by_rank[q][rank] = {item, b};
            seen[q] += 1;
        }
    }
    for (int64_t q = 0; q < nslot; ++q) {
        int rk = 0;
        const int cg = (int)(q / sc.nB);
        const int nw = j_writers(sc, (int)(q % sc.nB), cg / sc.G, cg % sc.G, 0, 0, &rk);
        if (seen[q] != nw) return 2;
        for (int r = 1; r < nw; ++r) {
            const auto &cur = by_rank[q][r], &prev = by_rank[q][r - 1];
            if (sc.cyclic ? !(prev.second > cur.second) : !(prev.first < cur.first)) return 3;
        }
    }
    if (info) {
        info[0] = pl.nB;
        info[1] = pl.C;
        info[2] = pl.Bc;
        info[3] = pl.cyclic ? 1 : 0;
        info[4] = pl.grid;
        info[5] = pl.G;
    }
    return MH_OK;
}

}  // namespace mh
