// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mh.h"

struct mh_mlp;

namespace mh {

constexpr int kPad = 256;          // particle arrays are padded to a multiple of this
constexpr double kFarAway = 1.0e6;  // position of padding bodies (mass 0)

inline int64_t pad_to(int64_t n, int64_t q) { return (n + q - 1) / q * q; }

// Thread-local last-error message (mh_last_error).
void set_error(const std::string &msg);

// NVTX range over the host-side issue of one phase of a step ("mh_step",
// "mh:predict", "mh:evaluate", "mh:correct", ...), so that a profiler can
// select kernels by phase (ncu --nvtx --nvtx-include "mh:evaluate/").  Without
// an attached tool a range costs a few nanoseconds.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

// Host-side fault injection for tests of the error paths: true when the
// comma-separated environment variable MH_FAULT lists `what` (alloc, launch,
// timeout, nonfinite).  No fault is ever made on the device.
bool fault_armed(const char *what);
int injected_step_fault(const char *fn);    // MH_ECUDA (launch), MH_ETIMEOUT (timeout) or MH_OK

// Record a CUDA failure and return MH_ECUDA (or MH_ENOMEM for allocations).
int cuda_fail(cudaError_t e, const char *what);

#define MH_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return mh::cuda_fail(e_, #call); \
    } while (0)

#define MH_LAUNCHED(what)                               \
    do {                                                \
        cudaError_t e_ = cudaGetLastError();            \
        if (e_ != cudaSuccess) return mh::cuda_fail(e_, what); \
    } while (0)

// Work decomposition of one O(N^2) evaluation: i-tiles x j-chunks.  Every
// (i-tile, j-chunk) item writes its own slot of a partial-sum buffer, and the
// corrector adds the S slots in a fixed order, so results do not depend on
// which CTA ran which item.
struct PairPlan {
    int threads;        // threads per CTA (one i per thread)
    int i_per_cta;      // i-particles per CTA tile
    int tj;             // j-records per shared-memory tile
    int split;          // S: number of j-chunks
    int grid;           // CTAs launched (each loops over items)
    int64_t n_itiles;
    int64_t chunk;      // j-records per chunk (multiple of tj)
    int ipt = 1;        // FP32 form: i-bodies per thread (1 or 2)
    bool packed = false;  // FP32 form: the two i-bodies of a thread share paired FP32 instructions
};

// Time-symmetric variable shared step (Section 3.3): dt = dir (H- + H+)/2 with
// H = eta w^(-1/2) (Eq. 24), w the maximum over pairs of G (m_i + m_j) s^(-3/2).
// The evaluations write w into device words; the predictor and corrector read
// them and compute dt on the device, so a step needs no host round trip.
constexpr int kTsMaxIter = 64;       // words per bank (one per evaluation of a step)
struct TimeSymArgs {
    unsigned long long *w = nullptr; // [2][kTsMaxIter] bit patterns of w, by bank and pass; null: constant dt
    double *t = nullptr;             // simulation time (device)
    int prev = 0;                    // index into w of the evaluation that gives this step's H-
    int bank = 0;                    // this step's evaluations write w[bank * kTsMaxIter + pass]
    int pass = 0;                    // corrector: the evaluation it follows
    int n_iter = 0;                  // passes of this step (the predictor clears that many words)
    double eta = 0.0, dir = 1.0;
};

// Device buffers of one simulation (every per-particle array is padded to Np).
struct DeviceState {
    int64_t N = 0, Np = 0;
    int p = 0;             // order 2(p+1)
    double *m = nullptr;   // [Np]
    double *x0 = nullptr, *v0 = nullptr;   // [3][Np] committed state at t0
    double *d0 = nullptr;  // [2p][3][Np]    a^(0..2p-1) at t0
    double *x1 = nullptr, *v1 = nullptr;   // [3][Np] current estimate at t1
    double *jrec = nullptr;   // FP64 evaluation input, [3(P+1)][Np] with P = max(p, 2p-1 for init)
    float *jrec32 = nullptr;  // FP32-pair evaluation input, [NF32][Np]
    double *part = nullptr;   // [S][P+1][3][Np] partial sums of the split-j evaluation
    size_t part_doubles = 0;  // capacity of part
    double *diag = nullptr;   // diagnostics scratch (energy partials, ecc rows, result)
    int *flag = nullptr;      // device status word (non-finite detection)
    // Precision form: bounds on |x| and |v| (IEEE bit patterns of non-negative
    // doubles, so integer atomicMax orders them) in two slots [slot][x, v].
    // A kernel writing the split input reads slot `flip` and raises slot
    // 1 - flip, so every thread of one kernel sees the same grid.
    unsigned long long *bound = nullptr;
    int flip = 0;
    // Precision form: source bodies whose pairs are evaluated in FP64.
    int n_heavy = 0;
    int *heavy = nullptr;     // [n_heavy] body indices (device)
    // Block time steps: per-body tick and level, the active list, and the
    // device words [next block tick, active count] read back once per block step.
    long long *T = nullptr;
    int *level = nullptr;
    int *act = nullptr;
    unsigned long long *blk = nullptr;
    unsigned long long *blk_host = nullptr;   // pinned host mirror of blk
    long long T_now = 0;
    // Time-symmetric variable steps: [2][kTsMaxIter] words of Eq. 24, the device
    // clock, and the index of the word holding the next step's H-.
    unsigned long long *tsw = nullptr;
    double *tst = nullptr;
    int ts_prev = 0;
    // Compensated summation (Section 3.2): [6][Np] carried compensation of x, v.
    double *comp = nullptr;
    // Pair-symmetric evaluation: the item counter and the per-(chunk, block)
    // write counters of its ordered j-side accumulation (all 0 between launches).
    unsigned *symsync = nullptr;
    size_t symsync_words = 0;
};

constexpr int kMaxHeavy = 32;

// Bits of the device status word (DeviceState::flag).
constexpr int kFlagNonFinite = 1;   // a step produced a non-finite position or velocity
constexpr int kFlagSymWait = 2;     // a pair-symmetric evaluation's bounded wait ran out
// Smallest padded body count for which symmetric = 1 picks the pair-symmetric
// kernel (16 blocks of 128 bodies, 144 block pairs).
constexpr int64_t kSymMinNp = 2048;
// Below this many bodies the O(N) step kernels run one warp per block and the
// FP64 evaluation's j-chunk partial sums are pre-added in parallel.
constexpr int64_t kSmallN = 8192;

}  // namespace mh

struct mh_sim {
    mh_config cfg;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_free;
    double eps = 0.0;
    double t = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    mh::DeviceState s;
    mh_counters ctr{};
    void *batch = nullptr;        // batched integrator bookkeeping (batch.cu), or null
    // learned predictor (optional): network, feature/output buffers, saved state for sampling
    mh_mlp *mlp = nullptr;
    float *lfeat = nullptr, *lout = nullptr;
    double *lsave = nullptr;      // x0, v0, d0 copies for mh_collect_samples
    unsigned long long *conv = nullptr, *conv_host = nullptr;
    // time-symmetric steps: CUDA graphs of two consecutive steps, by (n_iter, backward)
    std::map<std::pair<int, int>, cudaGraphExec_t> ts_graphs;
    std::map<std::pair<int, int>, mh_counters> ts_graph_inc;   // counter increments of one replay
};

namespace mh {

// Simulation construction (api.cu): allocate, upload, optionally initialise.
int create_shell(mh_sim **out, int64_t N, int order, const double *m, const double *x,
                 const double *v, double eps, const mh_config *cfg, void *stream, bool init);
int mh_create_shell(mh_sim **out, int64_t N, int order, const double *m, const double *x,
                    const double *v, double eps, const mh_config *cfg, void *stream);
void free_batch(mh_sim *sim);

// ---- kernels' host launchers (integrator.cu, pair.cu, diag.cu) ----

// Evaluation: fills part[0..S) with a^(0..P) partial sums of bodies i0 <= i < i1
// from bodies 0 <= j < n_j.  Input rows have stride ld: jrec (FP64, 3(P+1) rows)
// with masses m, or jrec32 (precision form, nf32(P) rows, mass last).
// ilist (optional, device): position i in [i0, i1) evaluates body ilist[i]; the
// partial sums are stored by position.
// wmax (optional, device, FP64 and P <= 3): raised to the maximum over pairs of
// G (m_i + m_j) s^(-3/2) as a bit pattern (Section 3.3, Eq. 24).
int launch_pair(int P, int precision, int64_t n_j, int64_t ld, const double *m, const double *jrec,
                const float *jrec32, double eps, double G, int64_t i0, int64_t i1, double *part,
                int64_t part_ld, const PairPlan &plan, cudaStream_t st, const int *ilist = nullptr,
                unsigned long long *wmax = nullptr);

// O(N) step kernels (integrator.cu): phase 0 = predict, 1 = correct.
int launch_step_phase(const DeviceState &s, const mh_config &cfg, double dt, int phase, bool last,
                      int split, cudaStream_t st, unsigned long long *conv = nullptr,
                      const TimeSymArgs *ts = nullptr);
int launch_collect(const DeviceState &s, double dt, const double *x0s, const double *v0s, const double *d0s,
                   float *feats, float *targ, cudaStream_t st);
int launch_learned_features(const DeviceState &s, double dt, float *feats, cudaStream_t st);
int launch_learned_apply(const DeviceState &s, const mh_config &cfg, double dt, const float *y, float clamp,
                         cudaStream_t st);
// MLP inference (mlp.cu)
int mlp_infer(mh_mlp *n, const float *X, float *Y, int64_t rows, cudaStream_t st);
int mlp_dims(const mh_mlp *n, int *n_in, int *n_out);
int launch_init_rows(const DeviceState &s, int have, cudaStream_t st);
int launch_block_init(const DeviceState &s, const mh_config &cfg, cudaStream_t st);
int launch_block_schedule(const DeviceState &s, const mh_config &cfg, cudaStream_t st);
// part_ld: row stride of the active bodies' partial sums (by active position);
// 0 = the padded body count.
int launch_block_phase(const DeviceState &s, const mh_config &cfg, long long T_next, int64_t n_act,
                       int phase, bool last, int split, cudaStream_t st, int64_t part_ld = 0);
int launch_init_reduce(const DeviceState &s, int nr, int lo, int hi, int split, cudaStream_t st);
// Small systems: slot 0 of s.part <- sum of its first `split` slots (rows nr).
int launch_reduce_slots(const DeviceState &s, int nr, int split, cudaStream_t st);
// Slot 0 of part (n positions, rows nr of stride ld) <- sum of its first `split`
// slots, one warp per (row, position), in a fixed order.
int launch_reduce_slots_warp(int64_t n, int64_t ld, int nr, int split, double *part, cudaStream_t st);
int launch_gather_active(int64_t n_act, int64_t Np, int nr, int split, const double *part, const int *act,
                         int64_t ld_out, double *out, cudaStream_t st);
int launch_reduce_out(int64_t n, int64_t ld_part, int nr, int split, const double *part, double *out,
                      cudaStream_t st);
int launch_split32(int64_t N, int P, const double *traj, const double *m, double G, float *rows,
                   unsigned long long *bound, cudaStream_t st);

// Hi/lo split of the precision form.  All hi parts lie on one power-of-two
// grid g with 2^23 g > 2 * bound, so hi_j - hi_i is exact in FP32 for every
// pair; lo = x - hi (|lo| <= g/2) carries the remaining bits.  A body beyond
// twice the bound still splits exactly (x = hi + lo to FP32 precision of lo),
// only its hi differences may round.
__host__ __device__ inline double split_grid(double bound)
{
    int e = 0;
    frexp(fmax(2.0 * bound, 2.2250738585072014e-308), &e);   // 2^(e-1) <= 2*bound < 2^e
    return ldexp(1.0, e - 23);
}

__device__ inline void split_hi_lo(double x, double g, double inv_g, float &hi, float &lo)
{
    const double h = rint(x * inv_g) * g;
    hi = (float)h;
    lo = (float)(x - (double)hi);
}

// Diagnostics (diag.cu): energy into *e_dev (device scalar); ecc rows [3][ld].
int launch_energy(const DeviceState &s, double eps, double G, double *scratch, double *e_dev,
                  cudaStream_t st);
int launch_ecc(const DeviceState &s, double G, int central, double *ecc, cudaStream_t st);
size_t energy_scratch_doubles(int64_t N);

// Short active lists: one warp per (body, j-chunk), lanes over the sources.
// plan_short gives the number of j-chunks (partial-sum slots); launch_pair_short
// fills slots [0, split) of part (rows (P+1)*3 of stride part_ld, by active
// position) for P = 1 .. 3 in either form.
constexpr int64_t kShortActive = 256;
int plan_short(int64_t n_i, int64_t n_j, int device);
int launch_pair_short(int P, int precision, int64_t n_i, int64_t n_j, int64_t ld, const double *m,
                      const double *jrec, const float *jrec32, double eps, double G, double *part,
                      int64_t part_ld, int split, const int *ilist, cudaStream_t st);

// FP32 form variant: 1 = one i-body per thread, 2 = two, 3 = two in packed FP32x2 lanes.
PairPlan plan_pair(int P, int precision, int64_t n_i, int64_t n_j, int split_hint, int device, int variant = 1);

// All-pairs FP64 evaluation that computes each unordered pair once (pair_sym.cu),
// P = 1 .. 5 (the precision form's, P = 1 .. 3).
// Valid (nB > 0) when ld is a positive multiple of its 128-body block; writes
// `slots` = C (1 + G) partial-sum slots of (P+1)*3 rows of stride ld, every one
// of them in full: C i-side slots (one per row chunk) and C G j-side slots (per
// row chunk and chain), each accumulated by several rows in a fixed order.
struct SymPlan {
    int nB = 0, D = 0, C = 0, Bc = 0;   // blocks, distances, row chunks, distances per chunk
    int G = 1;                          // accumulation chains per chunk (writer rows by row mod G)
    int K = 1;                          // rows per item (FP32-pair: one CTA of 2K warps sweeps K rows)
    int items = 0;                      // ceil(nB / K) C
    int grid = 0;
    bool cyclic = false;                // one item per CTA, all resident (else items handed out in row order)
    int slots = 0;                      // C (1 + G)
    int sync_words = 0;                 // 1 + C G nB counters of the ordered accumulation
};
SymPlan plan_sym(int P, int64_t ld, int device, bool fp32 = false);
// The same plan for a given number of resident CTAs (host only).
SymPlan plan_sym_slots(int64_t ld, int slots, bool fp32, int kmax);
// Checks of a plan's ordered accumulation (mh_sym_schedule_check).
int sym_schedule_check(int64_t ld, int slots, bool fp32, int *info);
// Device words of the ordered accumulation: `words` holds sync_words counters,
// all 0 between launches (a launch leaves them so); `flag` the simulation's
// status word, in which a wait that runs out after wait_ns sets kFlagSymWait.
// bias (0 in normal use) is added to every awaited count: the host's fault
// injection sets it so that the waits cannot end and must run out.
struct SymSync {
    unsigned *words = nullptr;
    int *flag = nullptr;
    unsigned long long wait_ns = 4000000000ull;
    unsigned bias = 0;
};
// The precision form's pair-symmetric evaluation (FP32 pairs, FP64 sums), same
// plan and slots; jrec32 as written by the step kernels (mass row holding G m).
int launch_pair_sym32(int P, const SymPlan &plan, const SymSync &sync, const float *jrec32, int64_t ld,
                      int64_t N, double eps, double *part, cudaStream_t st);
// wmax (optional, device): raised to the maximum over pairs of G (m_i + m_j) s^(-3/2)
// as a bit pattern (the time-step criterion of Section 3.3, Eq. 24).
int launch_pair_sym(int P, const SymPlan &plan, const SymSync &sync, const double *jrec, const double *m,
                    int64_t ld, int64_t N, double eps, double G, double *part, cudaStream_t st,
                    unsigned long long *wmax = nullptr);

// FP64 contributions of the heavy source bodies to every body i < N, written
// to partial slot `slot` (rows (P+1)*3 of stride part_ld, 0 = ld) of part.
int launch_pair_heavy(int P, int64_t N, int64_t ld, const double *m, const double *jrec,
                      const int *heavy, int n_heavy, double eps, double G, double *part, int slot,
                      cudaStream_t st, const int *ilist = nullptr, int64_t part_ld = 0);

// Number of FP32 rows of the precision-form evaluation input for a given P.
__host__ __device__ constexpr int nf32(int P) { return 12 + 3 * (P >= 2) + 3 * (P >= 3) + 1; }

}  // namespace mh
