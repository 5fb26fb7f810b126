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
// Both forms run K rows of one chunk per CTA, one CTA per SM, and one
// accumulation chain (G = 1): FP64 K = 3 (2 above P = 3), FP32-pair K = 6 where
// six rows' shared memory fits, else 4.  The turn computation takes any G
// (rows split into chains by row mod G); the plans use G = 1.

// Schedule of one launch (from SymPlan) and the ordered-accumulation words.
struct SymSched {
    int nB, D, C, Bc;
    int G;                 // accumulation chains per j-slot: writer rows are split by row mod G
    int K;                 // rows per item (rows qK .. qK + K - 1 of one chunk)
    int cyclic;            // 1: one item per CTA, all resident; writers by descending distance
    int items;             // ceil(nB / K) * C
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

// Distances [lo, hi) of the off-diagonal blocks of row chunk ch.
__host__ __device__ __forceinline__ void chunk_range(const SymSched &sc, int ch, int &lo, int &hi)
{
    lo = ch * sc.Bc > 1 ? ch * sc.Bc : 1;
    hi = ch * sc.Bc + sc.Bc < sc.D + 1 ? ch * sc.Bc + sc.Bc : sc.D + 1;
}

// Whether row J - b (mod nB) adds into j-slot (ch, g, J) at distance b (a
// distance of chunk ch), i.e. evaluates that block and is in chain g; *before:
// whether it comes before row I (which evaluates J at distance bI) in the
// accumulation order.
__host__ __device__ __forceinline__ bool j_writer(const SymSched &sc, int J, int g, int b, int I, int bI,
                                                  bool *before)
{
    int r = J - b;
    if (r < 0) r += sc.nB;
    if ((sc.nB & 1) == 0 && b == sc.D && r >= sc.nB / 2) return false;   // rows >= nB/2 skip distance nB/2
    if (r % sc.G != g) return false;
    *before = sc.cyclic ? (b > bI) : (r < I);
    return true;
}

// The rows that add into j-slot (ch, g, J): I' = J - b (mod nB) for the
// distances b >= 1 of chunk ch that row I' evaluates, with I' = g (mod G).
// Returns how many there are and, in *rank, how many of them come before row I
// (which evaluates J at distance bI).  One thread.
__host__ __device__ __forceinline__ int j_writers(const SymSched &sc, int J, int ch, int g, int I, int bI,
                                                  int *rank)
{
    int lo, hi, nw = 0, rk = 0;
    chunk_range(sc, ch, lo, hi);
    for (int b = lo; b < hi; ++b) {
        bool before = false;
        if (j_writer(sc, J, g, b, I, bI, &before)) {
            ++nw;
            rk += before;
        }
    }
    *rank = rk;
    return nw;
}

// The same count by the 32 lanes of one warp (each lane takes every 32nd
// distance); every lane gets the result.
__device__ __forceinline__ int j_writers_warp(const SymSched &sc, int J, int ch, int g, int I, int bI, int *rank)
{
    int lo, hi, nw = 0, rk = 0;
    chunk_range(sc, ch, lo, hi);
    const int lane = threadIdx.x & 31;
    for (int b0 = lo; b0 < hi; b0 += 32) {
        bool before = false;
        const bool wr = b0 + lane < hi && j_writer(sc, J, g, b0 + lane, I, bI, &before);
        nw += __popc(__ballot_sync(0xffffffffu, wr));
        rk += __popc(__ballot_sync(0xffffffffu, wr && before));
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
    int item, rank, next, ready;
    unsigned zero;        // bit g: j-slot (ch, g) of the item's own block has no writer
};

// Warp 0 at the start of item (I, ch): which of block I's j-slots of chunk ch
// no row adds into (they must hold zeros).
__device__ __forceinline__ unsigned unwritten_chains(const SymSched &sc, int I, int ch)
{
    unsigned z = 0;
    for (int g = 0; g < sc.G; ++g) {
        int rk;
        if (j_writers_warp(sc, I, ch, g, I, 0, &rk) == 0) z |= 1u << g;
    }
    return z;
}

// j-slot of chunk ch, chain g (the i-side slots come first).
__host__ __device__ __forceinline__ int64_t j_slot(const SymSched &sc, int ch, int g)
{
    return (int64_t)sc.C + (int64_t)ch * sc.G + g;
}

// Warp 0 of a row's threads (tu: thread index within the row) before row I's
// ordered flush into j-slot (ch, I mod G, J): publish the rank (0: this row
// writes first) and whether the turn has come (one look).
__device__ __forceinline__ void flush_rank(const SymSched &sc, FlushSmem &fs, int tu, int I, int J, int ch, int b)
{
    if (tu < 32) {
        const int g = I % sc.G;
        int rank = 0;
        const int nw = j_writers_warp(sc, J, ch, g, I, b, &rank);
        if (tu == 0) {
            fs.rank = rank;
            fs.next = rank + 1 == nw ? 0 : rank + 1;
            fs.ready = rank == 0 ||
                       ld_acquire(&sc.count[(j_slot(sc, ch, g) - sc.C) * sc.nB + J]) == (unsigned)rank + sc.bias;
        }
    }
}

// The row's thread 0: wait (bounded) for the turn flush_rank published, unless it had come.
__device__ __forceinline__ void flush_wait(const SymSched &sc, FlushSmem &fs, int tu, int I, int J, int ch)
{
    if (tu == 0 && !fs.ready) {
        wait_turn(&sc.count[(j_slot(sc, ch, I % sc.G) - sc.C) * sc.nB + J], (unsigned)fs.rank + sc.bias, sc);
        fs.ready = 1;
    }
}

// The row's thread 0 after the row's stores of the flush (behind the row's
// barrier): pass the turn on with a release store, which orders the row's
// stores before it (the last writer leaves the counter at 0).
__device__ __forceinline__ void flush_end(const SymSched &sc, const FlushSmem &fs, int tu, int I, int J, int ch)
{
    if (tu == 0)
        st_release(&sc.count[(j_slot(sc, ch, I % sc.G) - sc.C) * sc.nB + J], (unsigned)fs.next);
}

// Barrier of the n threads of row u of an item (barrier 0 is __syncthreads).
__device__ __forceinline__ void row_sync(int u, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(u + 1), "r"(n) : "memory");
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

// Rows per CTA of the FP64 kernel: 12 warps per SM at P <= 3, 8 above (its
// registers).
template <int P>
__host__ __device__ constexpr int sym64_rows() { return P <= 3 ? 3 : 2; }

// kH: also track w = G (m_i + m_j) s^(-3/2) over all pairs i != j, whose maximum
// gives the time-step criterion of Section 3.3 (Eq. 24: H = eta w_max^(-1/2)).
// Non-negative doubles order as their bit patterns, so the maximum is an
// integer maximum (off the FP64 pipe) and the result does not depend on the
// order of the pairs.
//
// A CTA takes K = sym64_rows<P>() consecutive rows of one chunk (4 warps per
// row, one CTA per SM) and one accumulation chain, as the precision form's
// kernel below: the writer before a row is the previous row of the same CTA,
// which reaches the block one block earlier.  A row's warps meet at named
// barriers of their own; the rows of a CTA only at the item boundaries.
template <int P, bool kH>
__global__ void __launch_bounds__(kSymR * sym64_rows<P>(), 1) k_pair_fp64_sym(SymArgs<P> a)
{
    constexpr int NR = 3 * (P + 1);
    constexpr int K = sym64_rows<P>();
    const SymSched &sc = a.sc;
    unsigned long long wm = 0ull;
    __shared__ double accs_all[K][NR][kSymR];   // per row: j-side sums of the current block, by column
    __shared__ FlushSmem fsu[K];
    __shared__ int s_item;
    const int u = threadIdx.x / kSymR;           // this thread's row of the item
    const int tu = threadIdx.x % kSymR;          // thread within the row's four warps
    const int lane = tu & 31;
    const int w = tu >> 5;
    const int src = (lane + 1) & 31;      // ring: after t passes lane l holds j-lane (l + t) mod 32
    double(*accs)[kSymR] = accs_all[u];
    FlushSmem &fs = fsu[u];
    const bool even = (sc.nB & 1) == 0;
    for (int n = 0;; ++n) {
        if (threadIdx.x == 0) s_item = (int)min(next_item(sc, n), (unsigned)sc.items);
        __syncthreads();
        const int item = s_item;
        if (item >= sc.items) break;
        const int I = (item / sc.C) * K + u;
        const int ch = item % sc.C;
        const bool live = I < sc.nB;
        if (tu < 32) {
            const unsigned z = live ? unwritten_chains(sc, I, ch) : 0u;
            if (tu == 0) fs.zero = z;
        }
        const int64_t ib = (int64_t)(live ? I : 0) * kSymR + tu;
        double ri[P + 1][3], gmi;
        load_body<P>(a, ib, ri, gmi);
        double acci[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acci[k][c] = 0.0;
        __syncthreads();
        for (int g = 0; g < sc.G; ++g)
            if (live && (fs.zero >> g & 1u)) {
                // no row adds into this j-slot of the block: it holds zeros
                double *out = a.part + j_slot(sc, ch, g) * NR * a.ld + ib;
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
            }

        const int dmax = (even && I >= sc.nB / 2) ? sc.D - 1 : sc.D;
        const int b0 = ch * sc.Bc;
        const int b1 = min(b0 + sc.Bc, sc.D + 1);
        for (int b = b1 - 1; b >= b0; --b) {
            const bool active = live && b <= dmax;   // rows >= nB/2 skip distance nB/2
            if (b == 0) {
                if (!active) continue;
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
            if (!active) continue;                   // the row's four warps skip together
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
                row_sync(u, kSymR);
            }
            // ordered flush of block J's j-side sums into j-slot (ch, I mod G, J)
            flush_rank(sc, fs, tu, I, J, ch, b);
            flush_wait(sc, fs, tu, I, J, ch);
            row_sync(u, kSymR);
            const bool add = fs.rank > 0;
            double *out = a.part + j_slot(sc, ch, I % sc.G) * NR * a.ld + (int64_t)J * kSymR + tu;
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const double v = accs[q][tu];
                __stcg(out + q * a.ld, add ? __ldcg(out + q * a.ld) + v : v);
            }
            row_sync(u, kSymR);
            flush_end(sc, fs, tu, I, J, ch);
        }
        if (live) {
            double *out = a.part + (int64_t)ch * NR * a.ld + ib;
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) out[(3 * k + c) * a.ld] = acci[k][c];
        }
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
    SymLaunch(const SymLaunch &) = delete;
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
    return SymSched{pl.nB, pl.D, pl.C, pl.Bc, pl.G, pl.K, pl.cyclic ? 1 : 0, pl.items, sy.words, sy.words + 1,
                    sy.flag, sy.wait_ns, sy.bias};
}

template <int P>
int launch_sym(const SymPlan &pl, const SymSync &sy, const double *jrec, const double *m, int64_t ld, int64_t N,
               double eps, double G, double *part, unsigned long long *wmax, cudaStream_t st)
{
    SymArgs<P> a{jrec, m, ld, N, make_sched(pl, sy), eps * eps, G, part, wmax};
    const SymLaunch l(pl, kSymR * sym64_rows<P>(), st);
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

// Two warps per row of blocks: lane l of warp w holds the bodies of i-subtiles
// 2w and 2w + 1 in the two lanes of Blackwell's paired FP32 instructions
// (FFMA2/FMUL2/FADD2), so every j-record passed around the ring serves two
// pairs and one issue slot advances both.  The i-side sums are packed too; the
// j-side sum of a ring lane adds both pairs' terms in FP32.  FP32 sums cover
// one 128-body block (as the tiles of the ordered kernels) and are added to
// FP64 once per block.

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

// cp.async of 16 bytes from global to shared memory, bypassing L1 (the data
// were written by other CTAs).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Two warps per row of blocks, two i-bodies per lane; FP32 sums over one
// block.  A CTA takes K consecutive rows (one item: rows qK .. qK + K - 1 of
// one chunk), one pair of warps per row, and every row sweeps the chunk's
// distances from the largest down.  The writer before row I in the single
// accumulation chain is row I - 1 at the next larger distance: for all rows
// but the CTA's first it is a row of the same CTA, which reaches that block one
// block earlier.  The rows of a CTA meet only at the item boundaries (a row's
// two warps use a named barrier of their own), so a row that runs ahead waits
// on the turn counter as a row of another CTA would.  One CTA per SM: CTAs
// that share an SM progress at very different speeds and their rows drift
// apart by many blocks; within one CTA the drift stays small (measured at
// 65537 bodies: 5 % of the flushes wait, for under 1 % of the time).
//
// The flush of a block's j-side sums is deferred by one block: right after the
// block each row looks whether its turn has come and, if so, starts
// asynchronous copies of the j-slot into shared memory; after the next block
// the turn is waited for if it had not come, the copies have landed, the sums
// are added and stored, and the turn is passed on.  The slot's latency is thus
// hidden behind a block of pair arithmetic.  The i-side FP64 sums of the item
// live in shared memory.  Shared memory per CTA: K (2 + 2 + 2) NR 128 words
// (dynamic, up to 216 KB at K = 6, P = 3).
template <int P>
struct Smem32 {
    static constexpr int NR = 3 * (P + 1);
    static constexpr size_t accs = (size_t)2 * NR * kSymR * sizeof(float);     // per row: two blocks in flight
    static constexpr size_t sbuf = (size_t)NR * kSymR * sizeof(double);        // per row: the j-slot being flushed
    static constexpr size_t acc64 = (size_t)NR * kSymR * sizeof(double);       // per row: i-side FP64 sums
    static constexpr size_t per_row = accs + sbuf + acc64;
    static size_t bytes(int K) { return (size_t)K * per_row; }
};

template <int P, int K>
__global__ void __launch_bounds__(64 * K, 1) k_pair_fp32_sym(SymArgs32<P> a)
{
    constexpr int NF = Rec32s<P>::NF;
    constexpr int NR = 3 * (P + 1);
    using SM = Smem32<P>;
    const SymSched &sc = a.sc;
    extern __shared__ __align__(16) unsigned char smem32[];
    __shared__ FlushSmem fsu[K];
    __shared__ int pend_J[K];
    __shared__ int s_item;
    const int u = threadIdx.x >> 6;                // this thread's row of the item
    const int tu = threadIdx.x & 63;               // thread within the row's two warps
    const int lane = tu & 31;
    const int w = tu >> 5;
    const int src = (lane + 1) & 31;
    const int fc = 2 * tu;                         // the two j-slot columns this thread flushes
    float(*accs)[NR][kSymR] = reinterpret_cast<float(*)[NR][kSymR]>(smem32 + u * SM::per_row);
    double(*sbuf)[kSymR] = reinterpret_cast<double(*)[kSymR]>(smem32 + u * SM::per_row + SM::accs);
    double(*acc64s)[kSymR] = reinterpret_cast<double(*)[kSymR]>(smem32 + u * SM::per_row + SM::accs + SM::sbuf);
    FlushSmem &fs = fsu[u];
    const bool even = (sc.nB & 1) == 0;
    const float2 eps2 = f2(a.eps2);
    for (int n = 0;; ++n) {
        if (threadIdx.x == 0) s_item = (int)min(next_item(sc, n), (unsigned)sc.items);
        __syncthreads();
        const int item = s_item;
        if (item >= sc.items) break;
        const int I = (item / sc.C) * K + u;
        const int ch = item % sc.C;
        const bool live = I < sc.nB;
        if (tu < 32) {
            const unsigned z = live ? unwritten_chains(sc, I, ch) : 0u;
            if (tu == 0) fs.zero = z;
        }
        // the lane's two i-bodies, negated (differences become additions), packed
        float2 ni[NF - 1], gmi;
        {
            float r0[NF], r1[NF];
            const int64_t base = (int64_t)(live ? I : 0) * kSymR;
            load_body32<P>(a, base + (2 * w) * 32 + lane, r0);
            load_body32<P>(a, base + (2 * w + 1) * 32 + lane, r1);
#pragma unroll
            for (int q = 0; q < NF - 1; ++q) ni[q] = make_float2(-r0[q], -r1[q]);
            gmi = make_float2(r0[NF - 1], r1[NF - 1]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc64s[q][(2 * w + k) * 32 + lane] = 0.0;
        __syncthreads();
        if (live && (fs.zero & 1u)) {
            // no row adds into this block's j-slot of chunk ch: it holds zeros
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                double *out = a.part + j_slot(sc, ch, 0) * NR * a.ld + (int64_t)I * kSymR + tu + k * 64;
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
            }
        }

        bool pending = false, copied = false;
        int kb = 0;                                // accs buffer of the row's current block
        // copy this thread's two columns of the row's pending j-slot (the first
        // writer has nothing to copy)
        auto start_copy = [&]() {
            if (fs.rank > 0) {
                const double *src_slot = a.part + j_slot(sc, ch, 0) * NR * a.ld + (int64_t)pend_J[u] * kSymR + fc;
#pragma unroll
                for (int q = 0; q < NR; ++q) cp_async16(&sbuf[q][fc], src_slot + q * a.ld);
            }
            cp_async_commit();
        };
        // finish the rows' pending flushes (the whole CTA takes part): wait for the
        // turn where it had not come, add the copied slot, store, pass the turn on
        auto finish_flushes = [&]() {
            if (pending && tu == 0 && !fs.ready) {
                wait_turn(&sc.count[(j_slot(sc, ch, 0) - sc.C) * sc.nB + pend_J[u]], (unsigned)fs.rank + sc.bias, sc);
                fs.ready = 1;
            }
            row_sync(u, 64);
            if (pending) {
                if (!copied) start_copy();
                cp_async_commit_wait_all();
                const bool add = fs.rank > 0;
                const int pb = kb ^ 1;
                double *out = a.part + j_slot(sc, ch, 0) * NR * a.ld + (int64_t)pend_J[u] * kSymR + fc;
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    double2 v = make_double2((double)accs[pb][q][fc], (double)accs[pb][q][fc + 1]);
                    if (add) {
                        v.x += sbuf[q][fc];
                        v.y += sbuf[q][fc + 1];
                    }
                    __stcg(reinterpret_cast<double2 *>(out + q * a.ld), v);
                }
            }
            row_sync(u, 64);
            if (pending && tu == 0)
                st_release(&sc.count[(j_slot(sc, ch, 0) - sc.C) * sc.nB + pend_J[u]], (unsigned)fs.next);
            pending = false;
        };

        const int b0 = ch * sc.Bc;
        const int b1 = min(b0 + sc.Bc, sc.D + 1);
        const int dmax = (even && I >= sc.nB / 2) ? sc.D - 1 : sc.D;
        for (int b = b1 - 1; b >= b0; --b) {
            const bool diag = b == 0;                // the same for every row of the CTA
            const bool active = live && b <= dmax;   // rows >= nB/2 skip distance nB/2
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
                if (active) {
                    float rj[NF];
                    load_body32<P>(a, (int64_t)J * kSymR + js * 32 + lane, rj);
                    float accj[P + 1][3];
#pragma unroll
                    for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                        for (int c = 0; c < 3; ++c) accj[n2][c] = 0.0f;
#pragma unroll 2
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
                                for (int c = 0; c < 3; ++c)
                                    accj[n3][c] = __shfl_sync(0xffffffffu, accj[n3][c], src);
                        }
                    }
                    if (!diag) {
                        // each column is visited twice, by warp 0 and by warp 1: first at
                        // stage 0 (columns 0, 2) or 1 (columns 1, 3), second at stage 2 or 3
#pragma unroll
                        for (int n3 = 0; n3 <= P; ++n3)
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                float &cell = accs[kb][3 * n3 + c][js * 32 + lane];
                                cell = (jt < 2 ? 0.0f : cell) + accj[n3][c];
                            }
                    }
                }
                if (!diag) row_sync(u, 64);
            }
            if (active) {
#pragma unroll
                for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc64s[3 * n2 + c][(2 * w) * 32 + lane] += (double)acci[n2][c].x;
                        acc64s[3 * n2 + c][(2 * w + 1) * 32 + lane] += (double)acci[n2][c].y;
                    }
            }
            finish_flushes();
            if (!diag) {
                // take the turn for block J's j-side sums if it has come (within the
                // CTA it has: the row before swept this block one step ago); else
                // after the next block
                if (active && tu < 32) {
                    int rank = 0;
                    const int nw = j_writers_warp(sc, J, ch, 0, I, b, &rank);
                    if (tu == 0) {
                        fs.rank = rank;
                        fs.next = rank + 1 == nw ? 0 : rank + 1;
                        fs.ready = rank == 0 || ld_acquire(&sc.count[(j_slot(sc, ch, 0) - sc.C) * sc.nB + J]) ==
                                                    (unsigned)rank + sc.bias;
                        pend_J[u] = J;
                    }
                }
                row_sync(u, 64);
                if (active) {
                    copied = fs.ready;
                    if (copied) start_copy();
                    pending = true;
                    kb ^= 1;
                }
            }
        }
        finish_flushes();
        if (live) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int col = (2 * w + k) * 32 + lane;
                double *out = a.part + (int64_t)ch * NR * a.ld + (int64_t)I * kSymR + col;
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.ld] = acc64s[q][col];
            }
        }
    }
}

template <int P>
int launch_sym32(const SymPlan &pl, const SymSync &sy, const float *jrec32, int64_t ld, int64_t N, double eps,
                 double *part, cudaStream_t st)
{
    SymArgs32<P> a{jrec32, ld, N, make_sched(pl, sy), (float)(eps * eps), part};
    SymLaunch l(pl, 64 * pl.K, st);
    l.cfg.dynamicSmemBytes = Smem32<P>::bytes(pl.K);
    if (pl.K == 6)
        MH_CUDA(cudaLaunchKernelEx(&l.cfg, k_pair_fp32_sym<P, 6>, a));
    else
        MH_CUDA(cudaLaunchKernelEx(&l.cfg, k_pair_fp32_sym<P, 4>, a));
    return MH_OK;
}

}  // namespace

// The plan for `slots` resident CTAs (items of equal size; the chunk count with
// the fewest block-times on the busiest CTA).  One item per CTA when they all fit
// at once (distance order); otherwise the CTAs take items in row order, and rows
// at the end of a launch that is only just above one wave wait for the first
// rows (their blocks near the wrap-around come last in that order): count one
// wave more.  FP64: K = sym64_rows rows per item (4 warps each), one chain.
// FP32-pair: K rows per item (K = kmax or 4, whichever wastes less of the last
// wave; a CTA sweeps K blocks per step), one chain.
SymPlan plan_sym_slots(int64_t ld, int slots, bool fp32, int kmax)
{
    SymPlan pl{};
    if (ld % kSymR != 0 || ld < kSymR || slots < 1) return pl;
    pl.nB = (int)(ld / kSymR);
    pl.D = pl.nB / 2;
    const int nb = pl.D + 1;                        // blocks of the longest row
    double best = 1e300;
    const int Ks[2] = {kmax, 4};
    for (int ki = 0; ki < (fp32 && kmax != 4 ? 2 : 1); ++ki) {
        const int K = Ks[ki];
        const int64_t groups = (pl.nB + K - 1) / K;
        for (int C = 1; C <= nb; ++C) {
            const int Bc = (nb + C - 1) / C;
            if ((nb + Bc - 1) / Bc != C) continue;
            const int64_t items = groups * C;
            const bool cyclic = items <= slots;
            int64_t waves = cyclic ? 1 : (items + slots - 1) / slots;
            if (!cyclic && items < slots + nb) waves += 1;
            const double cost = (double)waves * (Bc + 1.0) * K * (1.0 + 0.005 * C);
            if (cost < best) {
                best = cost;
                pl.C = C;
                pl.Bc = Bc;
                pl.K = K;
                pl.cyclic = cyclic;
                pl.items = (int)items;
            }
        }
    }
    pl.grid = (int)(pl.cyclic ? pl.items : std::min(pl.items, slots));
    pl.G = 1;
    pl.slots = pl.C * (1 + pl.G);
    pl.sync_words = 1 + pl.C * pl.G * pl.nB;
    return pl;
}

SymPlan plan_sym(int P, int64_t ld, int device, bool fp32)
{
    if (ld % kSymR != 0 || ld < kSymR || P < 1 || P > (fp32 ? 3 : 5)) return SymPlan{};
    // resident CTAs per device (FP32-pair: SMs, one CTA of K rows each, and the
    // largest K whose shared memory fits), cached per (device, P, form)
    static int slot_cache[64][16] = {{0}};
    static int kmax_cache[64][16] = {{0}};
    const int ci = P + (fp32 ? 8 : 0);
    const bool cached = device >= 0 && device < 64;
    int slots = cached ? slot_cache[device][ci] : 0;
    int kmax = cached ? kmax_cache[device][ci] : 0;
    if (slots == 0) {
        int n_sm = 0, occ = 0;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (fp32) {
            kmax = 4;
            const void *fn6 = P == 1 ? (const void *)k_pair_fp32_sym<1, 6>
                            : P == 2 ? (const void *)k_pair_fp32_sym<2, 6> : (const void *)k_pair_fp32_sym<3, 6>;
            const void *fn4 = P == 1 ? (const void *)k_pair_fp32_sym<1, 4>
                            : P == 2 ? (const void *)k_pair_fp32_sym<2, 4> : (const void *)k_pair_fp32_sym<3, 4>;
            const size_t b6 = P == 1 ? Smem32<1>::bytes(6) : P == 2 ? Smem32<2>::bytes(6) : Smem32<3>::bytes(6);
            const size_t b4 = P == 1 ? Smem32<1>::bytes(4) : P == 2 ? Smem32<2>::bytes(4) : Smem32<3>::bytes(4);
            cudaFuncSetAttribute(fn4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b4);
            if (cudaFuncSetAttribute(fn6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b6) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn6, 64 * 6, b6) == cudaSuccess && occ >= 1)
                kmax = 6;
            cudaGetLastError();
            occ = 1;
        } else {
            const void *fn = P == 1 ? (const void *)k_pair_fp64_sym<1, false>
                           : P == 2 ? (const void *)k_pair_fp64_sym<2, false>
                           : P == 3 ? (const void *)k_pair_fp64_sym<3, false>
                           : P == 4 ? (const void *)k_pair_fp64_sym<4, false> : (const void *)k_pair_fp64_sym<5, false>;
            kmax = P <= 3 ? sym64_rows<3>() : sym64_rows<5>();
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSymR * kmax, 0);
        }
        slots = std::max(n_sm, 1) * std::max(occ, 1);
        if (cached) {
            slot_cache[device][ci] = slots;
            kmax_cache[device][ci] = kmax;
        }
    }
    return plan_sym_slots(ld, slots, fp32, kmax);
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
int sym_schedule_check(int64_t ld, int slots, bool fp32, int *info)
{
    const SymPlan pl = plan_sym_slots(ld, slots, fp32, fp32 ? 6 : sym64_rows<3>());
    if (pl.nB == 0) return MH_EINVAL;
    SymSched sc{pl.nB, pl.D, pl.C, pl.Bc, pl.G, pl.K, pl.cyclic ? 1 : 0, pl.items, nullptr, nullptr, nullptr, 0, 0};
    const bool even = (pl.nB & 1) == 0;
    const int64_t nslot = (int64_t)pl.C * pl.G * pl.nB;
    std::vector<int> seen(nslot, 0), nwv(nslot, -1);
    std::vector<std::vector<std::pair<int, int>>> by_rank(nslot);   // rank -> (item, distance)
    for (int item = 0; item < sc.items; ++item) {
        const int ch = item % sc.C;
        for (int u = 0; u < sc.K; ++u) {
            const int I = (item / sc.C) * sc.K + u;
            if (I >= sc.nB) continue;
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
    }
    for (int64_t q = 0; q < nslot; ++q) {
        int rk = 0;
        const int cg = (int)(q / sc.nB);
        const int nw = j_writers(sc, (int)(q % sc.nB), cg / sc.G, cg % sc.G, 0, 0, &rk);
        if (seen[q] != nw) return 2;
        for (int r = 1; r < nw; ++r) {
            const auto &cur = by_rank[q][r], &prev = by_rank[q][r - 1];
            // distance order: the writer before sweeps a larger distance (all items
            // resident); row order: it was handed out earlier, or it is an earlier
            // row of the same item, which sweeps the larger distance first
            const bool ok = sc.cyclic ? prev.second > cur.second
                                      : prev.first < cur.first || (prev.first == cur.first && prev.second > cur.second);
            if (!ok) return 3;
        }
    }
    if (info) {
        info[0] = pl.nB;
        info[1] = pl.C;
        info[2] = pl.Bc;
        info[3] = pl.cyclic ? 1 : 0;
        info[4] = pl.grid;
        info[5] = pl.G;
        info[6] = pl.K;
    }
    return MH_OK;
}

}  // namespace mh
