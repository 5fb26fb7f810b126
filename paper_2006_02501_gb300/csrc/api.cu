// Host side of the C ABI declared in include/mh.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <cstdlib>
#include <string>
#include <vector>

#include "common.cuh"

namespace mh {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

bool fault_armed(const char *what)
{
    const char *env = std::getenv("MH_FAULT");
    if (!env || !*env) return false;
    const std::string list = std::string(",") + env + ",";
    return list.find(std::string(",") + what + ",") != std::string::npos;
}

// The step faults a test can inject: a failed kernel launch, or a bounded
// device-side wait that ran out.  Checked before any work is queued, so the
// state is left as it was.
int injected_step_fault(const char *fn)
{
    if (fault_armed("launch")) {
        set_error(std::string(fn) + ": kernel launch failed (injected by MH_FAULT=launch)");
        return MH_ECUDA;
    }
    if (fault_armed("timeout")) {
        set_error(std::string(fn) + ": a bounded device-side wait ran out (injected by MH_FAULT=timeout)");
        return MH_ETIMEOUT;
    }
    return MH_OK;
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();   // clear the sticky-free allocation error
        return MH_ENOMEM;
    }
    return MH_ECUDA;
}

namespace {

// Order 2(p+1) -> p.  The paper's schemes are of arbitrary order (Section 2);
// the library builds orders 4 to 12.
int order_to_p(int order)
{
    return order == 4 ? 1 : order == 6 ? 2 : order == 8 ? 3 : order == 10 ? 4 : order == 12 ? 5 : 0;
}

template <typename T>
int dalloc(T **ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) return MH_OK;
    if (fault_armed("alloc")) {
        set_error("device allocation failed (injected by MH_FAULT=alloc)");
        return MH_ENOMEM;
    }
    MH_CUDA(cudaMalloc((void **)ptr, count * sizeof(T)));
    return MH_OK;
}

void free_state(DeviceState &s)
{
    void *ptrs[] = {s.m, s.x0, s.v0, s.d0, s.x1, s.v1, s.jrec, s.jrec32, s.part, s.diag, s.flag, s.bound,
                    s.heavy, s.T, s.level, s.act, s.blk, s.tsw, s.tst, s.comp, s.symsync};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (s.blk_host) cudaFreeHost(s.blk_host);
    s = DeviceState{};
}

// AoS (N x K x 3) host array -> SoA rows [K*3][ld] (padding columns filled with fill).
void to_soa(const double *src, int64_t N, int K, int64_t ld, std::vector<double> &dst, double fill)
{
    dst.assign((size_t)K * 3 * ld, fill);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c) dst[(size_t)(3 * k + c) * ld + i] = src[((size_t)i * K + k) * 3 + c];
}

void from_soa(const std::vector<double> &src, int64_t N, int K, int64_t ld, double *dst)
{
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c) dst[((size_t)i * K + k) * 3 + c] = src[(size_t)(3 * k + c) * ld + i];
}

// Make sure the partial-sum buffer holds `need` doubles.
int ensure_part(DeviceState &s, size_t need, cudaStream_t st)
{
    if (need <= s.part_doubles) return MH_OK;
    if (s.part) {
        MH_CUDA(cudaStreamSynchronize(st));
        cudaFree(s.part);
        s.part = nullptr;
        s.part_doubles = 0;
    }
    int rc = dalloc(&s.part, need);
    if (rc) return rc;
    s.part_doubles = need;
    return MH_OK;
}

// Make sure the ordered-accumulation counters of the pair-symmetric evaluation
// hold `words` words; new words start at 0 (the state between launches).
int ensure_symsync(DeviceState &s, size_t words, cudaStream_t st)
{
    if (words <= s.symsync_words) return MH_OK;
    if (s.symsync) {
        MH_CUDA(cudaStreamSynchronize(st));
        cudaFree(s.symsync);
        s.symsync = nullptr;
        s.symsync_words = 0;
    }
    if (int rc = dalloc(&s.symsync, words)) return rc;
    MH_CUDA(cudaMemsetAsync(s.symsync, 0, words * sizeof(unsigned), st));
    s.symsync_words = words;
    return MH_OK;
}

// Partial sums and counters of one pair-symmetric launch.  MH_FAULT=symwait
// (tests of the timeout path) makes every wait of the launch unsatisfiable and
// its limit 20 ms, so the launch ends with kFlagSymWait set.
int prepare_sym(mh_sim *sim, const SymPlan &sp, int extra_slots, int P, SymSync *sy)
{
    DeviceState &s = sim->s;
    if (int rc = ensure_part(s, (size_t)(sp.slots + extra_slots) * (P + 1) * 3 * s.Np, sim->stream)) return rc;
    if (int rc = ensure_symsync(s, (size_t)sp.sync_words, sim->stream)) return rc;
    sy->words = s.symsync;
    sy->flag = s.flag;
    if (fault_armed("symwait")) {
        sy->bias = 0x40000000u;
        sy->wait_ns = 20000000ull;
    }
    return MH_OK;
}

// Resolve the timing events of finished evaluation launches (waits for the stream).
int collect_timing(mh_sim *sim)
{
    if (sim->ev_pending.empty()) return MH_OK;
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    for (auto &pr : sim->ev_pending) {
        float ms = 0.0f;
        MH_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        sim->ctr.pair_kernel_ms += ms;
        sim->ctr.pair_kernel_timed += 1;
        sim->ev_free.push_back(pr);
    }
    sim->ev_pending.clear();
    return MH_OK;
}

int timed_event_pair(mh_sim *sim, std::pair<cudaEvent_t, cudaEvent_t> *out)
{
    if (!sim->ev_free.empty()) {
        *out = sim->ev_free.back();
        sim->ev_free.pop_back();
        return MH_OK;
    }
    MH_CUDA(cudaEventCreate(&out->first));
    MH_CUDA(cudaEventCreate(&out->second));
    return MH_OK;
}

// Autotuner of the precision-form evaluation: kernel variant (1 = one i-body
// per thread, 2 = two, 3 = two in packed FP32x2 lanes) per (P, number of
// evaluated bodies rounded up to a power of two, sources, device).  Variants 1
// and 2 give bit-identical sums, variant 3 differs by the rounding of its
// explicit multiply-adds.  The first evaluation of a class times each variant
// once with CUDA events and keeps the fastest.
std::map<std::tuple<int, int64_t, int64_t, int>, int> g_variant_cache;

int tuned_variant(mh_sim *sim, int P, int64_t n_i, const int *ilist, int *variant)
{
    DeviceState &s = sim->s;
    if (sim->cfg.fp32_variant >= 1 && sim->cfg.fp32_variant <= 3) {
        *variant = sim->cfg.fp32_variant;
        return MH_OK;
    }
    *variant = 1;
    if (n_i < 8192) return MH_OK;          // a single wave either way: keep one body per thread
    int64_t bucket = 1;
    while (bucket < n_i) bucket <<= 1;
    const auto key = std::make_tuple(P, bucket, s.N, sim->device);
    auto it = g_variant_cache.find(key);
    if (it != g_variant_cache.end()) {
        *variant = it->second;
        return MH_OK;
    }
    constexpr int kVariants = 3;
    cudaEvent_t ev[kVariants + 1];
    for (auto &e : ev) MH_CUDA(cudaEventCreate(&e));
    for (int v = 1; v <= kVariants; ++v) {
        const PairPlan pl = plan_pair(P, MH_PREC_FP32PAIR, n_i, s.N, sim->cfg.split_j, sim->device, v);
        if (int rc = ensure_part(s, (size_t)(pl.split + 1) * (P + 1) * 3 * s.Np, sim->stream)) return rc;
        MH_CUDA(cudaEventRecord(ev[v - 1], sim->stream));
        if (int rc = launch_pair(P, MH_PREC_FP32PAIR, s.N, s.Np, s.m, s.jrec, s.jrec32, sim->eps, sim->cfg.G, 0,
                                 n_i, s.part, s.Np, pl, sim->stream, ilist))
            return rc;
    }
    MH_CUDA(cudaEventRecord(ev[kVariants], sim->stream));
    MH_CUDA(cudaEventSynchronize(ev[kVariants]));
    float best = 0.0f;
    for (int v = 1; v <= kVariants; ++v) {
        float ms = 0.0f;
        MH_CUDA(cudaEventElapsedTime(&ms, ev[v - 1], ev[v]));
        sim->ctr.pair_tune_ms_x1000[v - 1] = (int32_t)(ms * 1000.0f);
        if (v == 1 || ms < best) {
            best = ms;
            *variant = v;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    g_variant_cache[key] = *variant;
    return MH_OK;
}

// One O(N^2) evaluation of a^(0..P) for all bodies into s.part; returns S via *split.
// wslot (optional, device, zeroed by the caller): raised to the maximum over
// pairs of G (m_i + m_j) s^(-3/2) (Eq. 24); FP64 pair-symmetric kernel only.
int evaluate(mh_sim *sim, int P, int precision, int *split, unsigned long long *wslot = nullptr)
{
    DeviceState &s = sim->s;
    if (wslot && (precision != MH_PREC_FP64 || P > 5)) {
        set_error("evaluate: the Eq. 24 maximum is tracked by the FP64 kernels for P <= 5 only");
        return MH_EINVAL;
    }
    // pair-symmetric kernel: always (symmetric = 2), or (symmetric = 1) once there
    // are 16 blocks of 128 bodies; below, its blocks are too few to fill the GPU
    const int sym_mode = sim->cfg.symmetric;
    if (precision == MH_PREC_FP64 && P <= 5 && (sym_mode == 2 || (sym_mode == 1 && s.Np >= kSymMinNp))) {
        const SymPlan sp = plan_sym(P, s.Np, sim->device);
        if (sp.nB > 0) {
            SymSync sy;
            int rc = prepare_sym(sim, sp, 0, P, &sy);
            if (rc) return rc;
            std::pair<cudaEvent_t, cudaEvent_t> ev{};
            if (sim->timing) {
                if ((rc = timed_event_pair(sim, &ev))) return rc;
                MH_CUDA(cudaEventRecord(ev.first, sim->stream));
            }
            rc = launch_pair_sym(P, sp, sy, s.jrec, s.m, s.Np, s.N, sim->eps, sim->cfg.G, s.part, sim->stream,
                                 wslot);
            if (rc) return rc;
            if (sim->timing) {
                MH_CUDA(cudaEventRecord(ev.second, sim->stream));
                sim->ev_pending.push_back(ev);
            }
            *split = sp.slots;
            sim->ctr.evaluations += 1;
            sim->ctr.pair_interactions += (double)s.N * (double)(s.N - 1);
            sim->ctr.kernel_launches += 1;
            return MH_OK;
        }
    }
    if (precision == MH_PREC_FP32PAIR && P <= 3 && sim->cfg.fp32_variant == 0 &&
        (sym_mode == 2 || (sym_mode == 1 && s.Np >= kSymMinNp))) {
        // precision form, each unordered pair once; the heavy bodies' FP64 pairs in the slot after
        const SymPlan sp = plan_sym(P, s.Np, sim->device, true);
        const bool heavy = s.n_heavy > 0;
        const int slots = sp.slots + (heavy ? 1 : 0);
        if (sp.nB > 0) {
            SymSync sy;
            int rc = prepare_sym(sim, sp, heavy ? 1 : 0, P, &sy);
            if (rc) return rc;
            std::pair<cudaEvent_t, cudaEvent_t> ev{};
            if (sim->timing) {
                if ((rc = timed_event_pair(sim, &ev))) return rc;
                MH_CUDA(cudaEventRecord(ev.first, sim->stream));
            }
            if ((rc = launch_pair_sym32(P, sp, sy, s.jrec32, s.Np, s.N, sim->eps, s.part, sim->stream))) return rc;
            if (sim->timing) {
                MH_CUDA(cudaEventRecord(ev.second, sim->stream));
                sim->ev_pending.push_back(ev);
            }
            if (heavy) {
                if ((rc = launch_pair_heavy(P, s.N, s.Np, s.m, s.jrec, s.heavy, s.n_heavy, sim->eps, sim->cfg.G,
                                            s.part, sp.slots, sim->stream)))
                    return rc;
                sim->ctr.kernel_launches += 1;
            }
            sim->ctr.pair_variant = 4;
            *split = slots;
            sim->ctr.evaluations += 1;
            sim->ctr.pair_interactions += (double)s.N * (double)(s.N - 1);
            sim->ctr.kernel_launches += 1;
            return MH_OK;
        }
    }
    int ipt = 1;
    if (precision == MH_PREC_FP32PAIR)
        if (int rc = tuned_variant(sim, P, s.N, nullptr, &ipt)) return rc;
    sim->ctr.pair_variant = ipt;
    std::pair<cudaEvent_t, cudaEvent_t> ev{};
    if (sim->timing) {
        if (int rc = timed_event_pair(sim, &ev)) return rc;
        MH_CUDA(cudaEventRecord(ev.first, sim->stream));
    }
    const PairPlan pl = plan_pair(P, precision, s.N, s.N, sim->cfg.split_j, sim->device, ipt);
    const bool heavy = precision == MH_PREC_FP32PAIR && s.n_heavy > 0;
    const int slots = pl.split + (heavy ? 1 : 0);
    int rc = ensure_part(s, (size_t)slots * (P + 1) * 3 * s.Np, sim->stream);
    if (rc) return rc;
    rc = launch_pair(P, precision, s.N, s.Np, s.m, s.jrec, s.jrec32, sim->eps, sim->cfg.G, 0, s.N,
                     s.part, s.Np, pl, sim->stream, nullptr, wslot);
    if (rc) return rc;
    if (sim->timing) {
        MH_CUDA(cudaEventRecord(ev.second, sim->stream));
        sim->ev_pending.push_back(ev);
    }
    if (heavy) {
        rc = launch_pair_heavy(P, s.N, s.Np, s.m, s.jrec, s.heavy, s.n_heavy, sim->eps, sim->cfg.G,
                               s.part, pl.split, sim->stream);
        if (rc) return rc;
        sim->ctr.kernel_launches += 1;
    }
    int out_slots = slots;
    if (precision == MH_PREC_FP64 && s.N < kSmallN && slots >= 4) {
        // small systems: pre-add the many j-chunk slots with one thread per (row, body)
        if ((rc = launch_reduce_slots(s, (P + 1) * 3, slots, sim->stream))) return rc;
        sim->ctr.kernel_launches += 1;
        out_slots = 1;
    }
    *split = out_slots;
    sim->ctr.evaluations += 1;
    sim->ctr.pair_interactions += (double)s.N * (double)(s.N - 1);
    sim->ctr.kernel_launches += 1;
    return MH_OK;
}

// a^(0..2p-1) at t0 from x0, v0 by explicit pair derivatives: passes of two
// orders each, the later passes using the derivatives found before (Section 3).
int initialise(mh_sim *sim)
{
    DeviceState &s = sim->s;
    const int K = 2 * s.p;
    for (int have = 0; have < K; have += 2) {
        const int P = have + 1;
        int rc = launch_init_rows(s, have, sim->stream);
        if (rc) return rc;
        int split = 0;
        rc = evaluate(sim, P, MH_PREC_FP64, &split);
        if (rc) return rc;
        rc = launch_init_reduce(s, (P + 1) * 3, have, std::min(P + 1, K), split, sim->stream);
        if (rc) return rc;
        sim->ctr.kernel_launches += 2;
    }
    sim->ctr.evaluations -= s.p;   // initialisation passes are not step evaluations
    sim->ctr.pair_interactions -= (double)s.p * (double)s.N * (double)(s.N - 1);
    return MH_OK;
}

// Time-symmetric steps: Eq. 24 at the committed positions x0, written to word
// kTsMaxIter of the Eq. 24 words (bank 1, pass 0), which becomes the next
// step's H-.  One P = 1 evaluation of the pair-symmetric kernel (its partial
// sums are scratch here).
int timesym_start(mh_sim *sim)
{
    DeviceState &s = sim->s;
    if (!s.tsw) return MH_OK;
    MH_CUDA(cudaMemsetAsync(s.tsw + kTsMaxIter, 0, sizeof(unsigned long long), sim->stream));
    if (int rc = launch_init_rows(s, 0, sim->stream)) return rc;
    int split = 0;
    if (int rc = evaluate(sim, 1, MH_PREC_FP64, &split, s.tsw + kTsMaxIter)) return rc;
    sim->ctr.evaluations -= 1;        // not a step evaluation
    sim->ctr.pair_interactions -= (double)s.N * (double)(s.N - 1);
    sim->ctr.kernel_launches += 1;
    s.ts_prev = kTsMaxIter;
    return MH_OK;
}

// Precision form: both bound slots <- max |x|, max |v| of host state arrays (N x 3).
int upload_bounds(DeviceState &s, const double *x, const double *v, cudaStream_t st)
{
    if (!s.bound) return MH_OK;
    double bx = 0.0, bv = 0.0;
    for (int64_t q = 0; q < 3 * s.N; ++q) {
        bx = std::max(bx, std::fabs(x[q]));
        bv = std::max(bv, std::fabs(v[q]));
    }
    unsigned long long h[4];
    std::memcpy(&h[0], &bx, 8);
    std::memcpy(&h[1], &bv, 8);
    h[2] = h[0];
    h[3] = h[1];
    MH_CUDA(cudaMemcpyAsync(s.bound, h, sizeof(h), cudaMemcpyHostToDevice, st));
    MH_CUDA(cudaStreamSynchronize(st));
    s.flip = 0;
    return MH_OK;
}

int check_handle(const mh_sim *sim)
{
    if (!sim) {
        set_error("NULL mh_sim handle");
        return MH_EINVAL;
    }
    return MH_OK;
}

}  // namespace

}  // namespace mh

using namespace mh;

extern "C" {

void mh_config_default(mh_config *cfg)
{
    if (!cfg) return;
    cfg->order = 8;
    cfg->beta_mode = MH_BETA_MODIFIED;
    cfg->precision = MH_PREC_FP64;
    cfg->step_mode = MH_STEP_SHARED;
    cfg->G = 1.0;
    cfg->eta = 0.1;
    cfg->dt_max = 1.0 / 32.0;
    cfg->k_max = 12;
    cfg->split_j = 0;
    cfg->symmetric = 1;
    cfg->fp32_variant = 0;
    cfg->compensated = 0;
    cfg->heavy_frac = 1e-3;
}

const char *mh_last_error(void) { return g_last_error.c_str(); }

int mh_sym_schedule_check(int64_t N, int slots, int precision, int *info)
{
    if (N < 1 || slots < 1 || (precision != MH_PREC_FP64 && precision != MH_PREC_FP32PAIR)) {
        set_error("mh_sym_schedule_check: N and slots must be positive, precision FP64 or FP32-pair");
        return MH_EINVAL;
    }
    return sym_schedule_check(pad_to(N, kPad), slots, precision == MH_PREC_FP32PAIR, info);
}

}  // extern "C"

// Allocate a simulation, upload m, x, v and (if initialise) compute the initial
// derivatives of one system of N bodies.
int mh::create_shell(mh_sim **out, int64_t N, int order, const double *m, const double *x,
                     const double *v, double eps, const mh_config *cfg, void *stream, bool init)
{
    if (!out) {
        set_error("mh_create: out is NULL");
        return MH_EINVAL;
    }
    *out = nullptr;
    set_error("");
    mh_config c;
    if (cfg) c = *cfg; else mh_config_default(&c);
    c.order = order;
    const int p = order_to_p(order);
    if (p == 0) { set_error("mh_create: order must be 4, 6, 8, 10 or 12"); return MH_EINVAL; }
    if (p > 3 && c.precision != MH_PREC_FP64) {
        set_error("mh_create: the FP32-pair form is built for orders 4 to 8");
        return MH_EINVAL;
    }
    if (N < 1 || !m || !x || !v) { set_error("mh_create: N >= 1 and non-NULL m, x, v required"); return MH_EINVAL; }
    if (!(eps >= 0.0) || !std::isfinite(eps)) { set_error("mh_create: eps must be finite and >= 0"); return MH_EINVAL; }
    if (c.precision != MH_PREC_FP64 && c.precision != MH_PREC_FP32PAIR) { set_error("mh_create: bad precision"); return MH_EINVAL; }
    if (c.beta_mode != MH_BETA_MODIFIED && c.beta_mode != MH_BETA_STANDARD) { set_error("mh_create: bad beta_mode"); return MH_EINVAL; }
    if (c.step_mode != MH_STEP_SHARED && c.step_mode != MH_STEP_BLOCK && c.step_mode != MH_STEP_TIMESYM) {
        set_error("mh_create: bad step_mode");
        return MH_EINVAL;
    }
    if (c.step_mode == MH_STEP_TIMESYM &&
        (c.precision != MH_PREC_FP64 || N < 2 || !(c.eta > 0.0) || !std::isfinite(c.eta))) {
        set_error("mh_create: time-symmetric steps need FP64, N >= 2 and a finite eta > 0");
        return MH_EINVAL;
    }
    if (c.symmetric < 0 || c.symmetric > 2) { set_error("mh_create: symmetric must be 0, 1 or 2"); return MH_EINVAL; }
    if (c.compensated != 0 && (c.compensated != 1 || c.step_mode != MH_STEP_SHARED)) {
        set_error("mh_create: compensated summation (compensated = 1) is built for shared constant steps");
        return MH_EINVAL;
    }
    if (c.fp32_variant < 0 || c.fp32_variant > 3) { set_error("mh_create: fp32_variant must be 0..3"); return MH_EINVAL; }
    if (c.step_mode == MH_STEP_BLOCK) {
        if (p < 2 || p > 3) { set_error("mh_create: block steps need order 6 or 8"); return MH_EINVAL; }
        if (!(c.dt_max > 0.0) || !std::isfinite(c.dt_max) || c.k_max < 0 || c.k_max > 30 || !(c.eta > 0.0)) {
            set_error("mh_create: block steps need dt_max > 0, 0 <= k_max <= 30, eta > 0");
            return MH_EINVAL;
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        if (!std::isfinite(m[i]) || m[i] < 0.0) { set_error("mh_create: masses must be finite and >= 0"); return MH_EINVAL; }
        for (int q = 0; q < 3; ++q)
            if (!std::isfinite(x[3 * i + q]) || !std::isfinite(v[3 * i + q])) { set_error("mh_create: non-finite x or v"); return MH_ENONFINITE; }
    }

    mh_sim *sim = new (std::nothrow) mh_sim();
    if (!sim) { set_error("mh_create: host allocation failed"); return MH_ENOMEM; }
    sim->cfg = c;
    sim->eps = eps;
    cudaGetDevice(&sim->device);
    if (stream && stream != (void *)cudaStreamLegacy && stream != (void *)cudaStreamPerThread) {
        sim->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { int rc = cuda_fail(e, "cudaStreamCreate"); delete sim; return rc; }
        sim->own_stream = true;
    }
    DeviceState &s = sim->s;
    s.N = N;
    s.Np = pad_to(N, kPad);
    s.p = p;
    const int K = 2 * p;
    const int Pinit = K - 1;                 // highest pair derivative of the initialisation
    const int rows64 = 3 * (std::max(Pinit, p) + 1);
    int rc = MH_OK;
    auto fail = [&](int r) { free_state(s); if (sim->own_stream) cudaStreamDestroy(sim->stream); delete sim; return r; };
    if ((rc = dalloc(&s.m, s.Np)) || (rc = dalloc(&s.x0, 3 * s.Np)) || (rc = dalloc(&s.v0, 3 * s.Np)) ||
        (rc = dalloc(&s.d0, (size_t)K * 3 * s.Np)) || (rc = dalloc(&s.x1, 3 * s.Np)) ||
        (rc = dalloc(&s.v1, 3 * s.Np)) || (rc = dalloc(&s.jrec, (size_t)rows64 * s.Np)) ||
        (rc = dalloc(&s.flag, 1)) || (rc = dalloc(&s.diag, 3 * s.Np + energy_scratch_doubles(N) + 1)))
        return fail(rc);
    if (c.precision == MH_PREC_FP32PAIR &&
        ((rc = dalloc(&s.jrec32, (size_t)nf32(p) * s.Np)) || (rc = dalloc(&s.bound, 4))))
        return fail(rc);
    if (c.step_mode == MH_STEP_BLOCK) {
        if ((rc = dalloc(&s.T, s.Np)) || (rc = dalloc(&s.level, s.Np)) || (rc = dalloc(&s.act, s.Np)) ||
            (rc = dalloc(&s.blk, 2)))
            return fail(rc);
        cudaError_t eh = cudaMallocHost((void **)&s.blk_host, 2 * sizeof(unsigned long long));
        if (eh != cudaSuccess) return fail(cuda_fail(eh, "cudaMallocHost"));
    }
    if (c.compensated) {
        if ((rc = dalloc(&s.comp, 6 * s.Np))) return fail(rc);
        cudaError_t ez = cudaMemsetAsync(s.comp, 0, 6 * s.Np * sizeof(double), sim->stream);
        if (ez != cudaSuccess) return fail(cuda_fail(ez, "cudaMemsetAsync"));
    }
    if (c.step_mode == MH_STEP_TIMESYM) {
        if ((rc = dalloc(&s.tsw, 2 * kTsMaxIter)) || (rc = dalloc(&s.tst, 1))) return fail(rc);
        cudaError_t ez = cudaMemsetAsync(s.tsw, 0, 2 * kTsMaxIter * sizeof(unsigned long long), sim->stream);
        if (ez == cudaSuccess) ez = cudaMemsetAsync(s.tst, 0, sizeof(double), sim->stream);
        if (ez != cudaSuccess) return fail(cuda_fail(ez, "cudaMemsetAsync"));
    }

    std::vector<double> h;
    h.assign(s.Np, 0.0);
    std::memcpy(h.data(), m, N * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(s.m, h.data(), s.Np * sizeof(double), cudaMemcpyHostToDevice, sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "copy m"));
    std::vector<double> hx, hv;
    to_soa(x, N, 1, s.Np, hx, 0.0);
    for (int c3 = 0; c3 < 3; ++c3)
        for (int64_t i = N; i < s.Np; ++i) hx[(size_t)c3 * s.Np + i] = kFarAway;
    to_soa(v, N, 1, s.Np, hv, 0.0);
    e = cudaMemcpyAsync(s.x0, hx.data(), 3 * s.Np * sizeof(double), cudaMemcpyHostToDevice, sim->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.v0, hv.data(), 3 * s.Np * sizeof(double), cudaMemcpyHostToDevice, sim->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d0, 0, (size_t)K * 3 * s.Np * sizeof(double), sim->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.jrec, 0, (size_t)rows64 * s.Np * sizeof(double), sim->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.flag, 0, sizeof(int), sim->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.x1, s.x0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.v1, s.v0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream);
    std::vector<float> m32;
    std::vector<int> heavy;
    if (e == cudaSuccess && s.jrec32) {
        // heavy source bodies: their pairs run in FP64, so their FP32 mass is 0
        double mtot = 0.0;
        for (int64_t i = 0; i < N; ++i) mtot += m[i];
        if (c.heavy_frac > 0.0)
            for (int64_t i = 0; i < N; ++i)
                if (m[i] > 0.0 && m[i] >= c.heavy_frac * mtot && (int)heavy.size() < kMaxHeavy)
                    heavy.push_back((int)i);
        // precision-form input: the mass row is constant, the others are written by every step
        e = cudaMemsetAsync(s.jrec32, 0, (size_t)nf32(p) * s.Np * sizeof(float), sim->stream);
        m32.assign(s.Np, 0.0f);
        for (int64_t i = 0; i < N; ++i) m32[i] = (float)(c.G * m[i]);
        for (int h : heavy) m32[h] = 0.0f;
        if (e == cudaSuccess && !heavy.empty()) {
            e = cudaMalloc((void **)&s.heavy, heavy.size() * sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.heavy, heavy.data(), heavy.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, sim->stream);
            s.n_heavy = (int)heavy.size();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.jrec32 + (size_t)(nf32(p) - 1) * s.Np, m32.data(), s.Np * sizeof(float),
                                cudaMemcpyHostToDevice, sim->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);   // host buffers go out of scope
    if (e != cudaSuccess) return fail(cuda_fail(e, "upload state"));
    if ((rc = upload_bounds(s, x, v, sim->stream))) return fail(rc);
    if (init) {
        if ((rc = initialise(sim))) return fail(rc);
        if (c.step_mode == MH_STEP_BLOCK && (rc = launch_block_init(s, c, sim->stream))) return fail(rc);
        if ((rc = timesym_start(sim))) return fail(rc);
    }
    e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "initialisation"));
    *out = sim;
    return MH_OK;
}

int mh::mh_create_shell(mh_sim **out, int64_t N, int order, const double *m, const double *x,
                        const double *v, double eps, const mh_config *cfg, void *stream)
{
    return create_shell(out, N, order, m, x, v, eps, cfg, stream, false);
}

extern "C" {

int mh_create(mh_sim **out, int64_t N, int order, const double *m, const double *x, const double *v,
              double eps, const mh_config *cfg, void *stream)
{
    return create_shell(out, N, order, m, x, v, eps, cfg, stream, true);
}

int mh_restore(mh_sim **out, int64_t N, int order, const double *m, const mh_state *state, double eps,
               const mh_config *cfg, void *stream)
{
    if (!out) { set_error("mh_restore: out is NULL"); return MH_EINVAL; }
    *out = nullptr;
    if (!state || !state->x || !state->v || !state->derivs) {
        set_error("mh_restore: the state needs x, v and derivs");
        return MH_EINVAL;
    }
    mh_sim *sim = nullptr;
    if (int rc = create_shell(&sim, N, order, m, state->x, state->v, eps, cfg, stream, false)) return rc;
    if (int rc = mh_set_state(sim, state)) {
        mh_destroy(sim);
        return rc;
    }
    *out = sim;
    return MH_OK;
}

void mh_destroy(mh_sim *sim)
{
    if (!sim) return;
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    free_batch(sim);
    for (auto &pr : sim->ev_pending) sim->ev_free.push_back(pr);
    for (auto &pr : sim->ev_free) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (sim->lfeat) cudaFree(sim->lfeat);
    if (sim->lout) cudaFree(sim->lout);
    if (sim->lsave) cudaFree(sim->lsave);
    if (sim->conv) cudaFree(sim->conv);
    if (sim->conv_host) cudaFreeHost(sim->conv_host);
    for (auto &kv : sim->ts_graphs) cudaGraphExecDestroy(kv.second);
    free_state(sim->s);
    if (sim->own_stream && sim->stream) cudaStreamDestroy(sim->stream);
    delete sim;
}

// Block steps with at least half the bodies due (or every block step with
// symmetric = 2): the pair-symmetric kernel evaluates all N bodies in N^2/2
// pair evaluations, against n_act N ordered ones for the active list alone.
static bool block_use_sym(const mh_sim *sim, int64_t n_act)
{
    const mh_config &c = sim->cfg;
    const DeviceState &s = sim->s;
    if (c.symmetric == 0 || (c.precision == MH_PREC_FP32PAIR && c.fp32_variant != 0)) return false;
    if (c.symmetric == 1 && (s.Np < kSymMinNp || 2 * n_act < s.N)) return false;
    return plan_sym(s.p, s.Np, sim->device, c.precision == MH_PREC_FP32PAIR).nB > 0;
}

// The n_iter evaluate-correct passes of one block step through the shared-step
// evaluation of all bodies (slots by body index), the active bodies' sums
// gathered in slot order into one compact slot after them, and the block
// corrector on that slot.
static int block_passes_sym(mh_sim *sim, long long T_next, int64_t n_act, int64_t part_ld, int n_iter)
{
    DeviceState &s = sim->s;
    const mh_config &c = sim->cfg;
    const int nr = (s.p + 1) * 3;
    const SymPlan sp = plan_sym(s.p, s.Np, sim->device, c.precision == MH_PREC_FP32PAIR);
    const size_t sym_doubles = (size_t)(sp.slots + 1) * nr * s.Np;     // + the heavy bodies' slot
    if (int rc = ensure_part(s, sym_doubles + (size_t)nr * part_ld, sim->stream)) return rc;
    for (int it = 0; it < n_iter; ++it) {
        int split = 0;
        if (int rc = evaluate(sim, s.p, c.precision, &split)) return rc;
        const size_t off = (size_t)split * nr * s.Np;
        if (off + (size_t)nr * part_ld > s.part_doubles) {
            set_error("mh_step: block step partial sums exceed their buffer");
            return MH_EINVAL;
        }
        if (int rc = launch_gather_active(n_act, s.Np, nr, split, s.part, s.act, part_ld, s.part + off,
                                          sim->stream))
            return rc;
        DeviceState sa = s;
        sa.part = s.part + off;
        const bool last = it == n_iter - 1;
        if (int rc = launch_block_phase(sa, c, T_next, n_act, 1, last, 1, sim->stream, part_ld)) return rc;
        if (!last) s.flip ^= 1;
        sim->ctr.kernel_launches += 3;
        // count the active bodies' interactions, as the ordered path does
        sim->ctr.pair_interactions += ((double)n_act - (double)s.N) * (double)(s.N - 1);
    }
    return MH_OK;
}

static int block_advance(mh_sim *sim, double dt, int n_iter)
{
    DeviceState &s = sim->s;
    const mh_config &c = sim->cfg;
    const double q = dt / c.dt_max;
    const long long nq = std::llround(q);
    if (!(dt > 0.0) || nq < 1 || std::fabs(q - (double)nq) > 1e-9 * std::max(1.0, q)) {
        set_error("mh_step: in block mode dt must be a positive multiple of dt_max");
        return MH_EINVAL;
    }
    const long long span0 = 1LL << c.k_max;
    const long long target = s.T_now + nq * span0;
    const int prec = c.precision;
    for (;;) {
        if (int rc = launch_block_schedule(s, c, sim->stream)) return rc;
        MH_CUDA(cudaMemcpyAsync(s.blk_host, s.blk, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                sim->stream));
        MH_CUDA(cudaStreamSynchronize(sim->stream));
        const long long T_next = (long long)s.blk_host[0];
        const int64_t n_act = (int64_t)s.blk_host[1];
        sim->ctr.kernel_launches += 3;
        if (n_act < 1 || T_next > target) {
            set_error("mh_step: block schedule out of order (levels corrupted?)");
            return MH_EINVAL;
        }
        if (int rc = launch_block_phase(s, c, T_next, n_act, 0, false, 0, sim->stream)) return rc;
        s.flip ^= 1;
        sim->ctr.kernel_launches += 1;
        int ipt = 1;
        if (prec == MH_PREC_FP32PAIR)
            if (int rc = tuned_variant(sim, s.p, n_act, s.act, &ipt)) return rc;
        sim->ctr.pair_variant = ipt;
        // partial sums by active position, rows of the padded active count
        const int64_t part_ld = pad_to(n_act, 32);
        if (block_use_sym(sim, n_act)) {
            // every unordered pair once for all bodies, then the active bodies' sums
            if (int rc = block_passes_sym(sim, T_next, n_act, part_ld, n_iter)) return rc;
            sim->ctr.particle_steps += (double)n_act;
            s.T_now = T_next;
            if (T_next == target) break;
            continue;
        }
        // a few bodies due: one warp per (body, j-chunk) over all the sources
        const bool short_list = n_act <= kShortActive && c.split_j == 0;
        for (int it = 0; it < n_iter; ++it) {
            const PairPlan pl = short_list ? PairPlan{} : plan_pair(s.p, prec, n_act, s.N, c.split_j, sim->device, ipt);
            const int split0 = short_list ? plan_short(n_act, s.N, sim->device) : pl.split;
            const bool heavy = prec == MH_PREC_FP32PAIR && s.n_heavy > 0;
            const int slots = split0 + (heavy ? 1 : 0);
            if (int rc = ensure_part(s, (size_t)slots * (s.p + 1) * 3 * part_ld, sim->stream)) return rc;
            std::pair<cudaEvent_t, cudaEvent_t> ev{};
            if (sim->timing) {
                if (int rc = timed_event_pair(sim, &ev)) return rc;
                MH_CUDA(cudaEventRecord(ev.first, sim->stream));
            }
            if (short_list) {
                if (int rc = launch_pair_short(s.p, prec, n_act, s.N, s.Np, s.m, s.jrec, s.jrec32, sim->eps, c.G,
                                               s.part, part_ld, split0, s.act, sim->stream))
                    return rc;
            } else if (int rc = launch_pair(s.p, prec, s.N, s.Np, s.m, s.jrec, s.jrec32, sim->eps, c.G, 0, n_act,
                                            s.part, part_ld, pl, sim->stream, s.act)) {
                return rc;
            }
            if (sim->timing) {
                MH_CUDA(cudaEventRecord(ev.second, sim->stream));
                sim->ev_pending.push_back(ev);
            }
            if (heavy) {
                if (int rc = launch_pair_heavy(s.p, n_act, s.Np, s.m, s.jrec, s.heavy, s.n_heavy, sim->eps, c.G,
                                               s.part, split0, sim->stream, s.act, part_ld))
                    return rc;
                sim->ctr.kernel_launches += 1;
            }
            const bool last = it == n_iter - 1;
            int split = slots;
            if (slots > 16 && n_act <= 4096) {
                // a short active list spread over many j-chunks: add the slots with
                // one warp per (row, body) instead of one thread
                if (int rc = launch_reduce_slots_warp(n_act, part_ld, (s.p + 1) * 3, slots, s.part, sim->stream))
                    return rc;
                sim->ctr.kernel_launches += 1;
                split = 1;
            }
            if (int rc = launch_block_phase(s, c, T_next, n_act, 1, last, split, sim->stream, part_ld)) return rc;
            if (!last) s.flip ^= 1;
            sim->ctr.kernel_launches += 2;
            sim->ctr.evaluations += 1;
            sim->ctr.pair_interactions += (double)n_act * (double)(s.N - 1);
        }
        sim->ctr.particle_steps += (double)n_act;
        s.T_now = T_next;
        if (T_next == target) break;
    }
    sim->t += dt;
    sim->ctr.steps += 1;
    return MH_OK;
}

// One shared step: P (plus the learned residual when a network is set), then
// E, C passes: exactly n_iter of them (tol < 0), or until the largest position
// change of a pass is at most tol * max|x| (at most n_iter passes).
static int shared_step(mh_sim *sim, double dt, int n_iter, double tol, int *n_used)
{
    DeviceState &s = sim->s;
    const int prec = sim->cfg.precision;
    int rc;
    {
        NvtxScope r("mh:predict");
        rc = launch_step_phase(s, sim->cfg, dt, 0, false, 0, sim->stream);
    }
    if (rc) return rc;
    s.flip ^= 1;                        // the predictor raised the other bound slot
    sim->ctr.kernel_launches += 1;
    if (sim->mlp) {
        if ((rc = launch_learned_features(s, dt, sim->lfeat, sim->stream))) return rc;
        if ((rc = mlp_infer(sim->mlp, sim->lfeat, sim->lout, s.N, sim->stream))) return rc;
        if ((rc = launch_learned_apply(s, sim->cfg, dt, sim->lout, 1e3f, sim->stream))) return rc;
        s.flip ^= 1;
        sim->ctr.kernel_launches += 9;
    }
    const bool adaptive = tol >= 0.0;
    int used = n_iter;
    for (int it = 0; it < n_iter; ++it) {
        int split = 0;
        {
            NvtxScope r("mh:evaluate");
            rc = evaluate(sim, s.p, prec, &split);
        }
        if (rc) return rc;
        NvtxScope rc_scope("mh:correct");
        bool last = it == n_iter - 1;
        if (adaptive) {
            MH_CUDA(cudaMemsetAsync(sim->conv, 0, 2 * sizeof(unsigned long long), sim->stream));
            if ((rc = launch_step_phase(s, sim->cfg, dt, 1, false, split, sim->stream, sim->conv))) return rc;
            s.flip ^= 1;
            MH_CUDA(cudaMemcpyAsync(sim->conv_host, sim->conv, 2 * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, sim->stream));
            MH_CUDA(cudaStreamSynchronize(sim->stream));
            double dx = 0.0, xm = 0.0;
            std::memcpy(&dx, &sim->conv_host[0], 8);
            std::memcpy(&xm, &sim->conv_host[1], 8);
            sim->ctr.kernel_launches += 1;
            if (dx <= tol * xm) last = true;
            if (last) {
                used = it + 1;
                // the converged pass again, now committing (same inputs, same result)
                if ((rc = launch_step_phase(s, sim->cfg, dt, 1, true, split, sim->stream))) return rc;
                sim->ctr.kernel_launches += 1;
                break;
            }
        } else {
            if ((rc = launch_step_phase(s, sim->cfg, dt, 1, last, split, sim->stream))) return rc;
            if (!last) s.flip ^= 1;
            sim->ctr.kernel_launches += 1;
        }
    }
    if (n_used) *n_used = used;
    sim->t += dt;
    sim->ctr.steps += 1;
    sim->ctr.particle_steps += (double)s.N;
    return MH_OK;
}

// One time-symmetric variable step (Section 3.3): P with dt = dir H-, then
// n_iter (E, C) passes; every E also finds Eq. 24's maximum at the positions
// it evaluates and the C after it uses dt = dir (H- + H+)/2.  The last E's word
// is the next step's H-.  dt and the clock stay on the device.
static int timesym_step(mh_sim *sim, int n_iter, double dir)
{
    DeviceState &s = sim->s;
    TimeSymArgs ts;
    ts.w = s.tsw;
    ts.t = s.tst;
    ts.prev = s.ts_prev;
    ts.bank = 1 - s.ts_prev / kTsMaxIter;
    ts.n_iter = n_iter;
    ts.eta = sim->cfg.eta;
    ts.dir = dir;
    int rc = launch_step_phase(s, sim->cfg, 0.0, 0, false, 0, sim->stream, nullptr, &ts);
    if (rc) return rc;
    sim->ctr.kernel_launches += 1;
    for (int it = 0; it < n_iter; ++it) {
        int split = 0;
        if ((rc = evaluate(sim, s.p, MH_PREC_FP64, &split, s.tsw + ts.bank * kTsMaxIter + it))) return rc;
        ts.pass = it;
        const bool last = it == n_iter - 1;
        if ((rc = launch_step_phase(s, sim->cfg, 0.0, 1, last, split, sim->stream, nullptr, &ts))) return rc;
        sim->ctr.kernel_launches += 1;
    }
    s.ts_prev = ts.bank * kTsMaxIter + n_iter - 1;
    sim->ctr.steps += 1;
    sim->ctr.particle_steps += (double)s.N;
    return MH_OK;
}

int mh_step_timesym(mh_sim *sim, int64_t nsteps, int n_iter, int backward)
{
    if (int rc = check_handle(sim)) return rc;
    if (sim->cfg.step_mode != MH_STEP_TIMESYM || !sim->s.tsw) {
        set_error("mh_step_timesym: the simulation was not created with step_mode MH_STEP_TIMESYM");
        return MH_EINVAL;
    }
    if (nsteps < 0 || n_iter < 1 || n_iter > kTsMaxIter) {
        set_error("mh_step_timesym: nsteps >= 0 and 1 <= n_iter <= 64 required");
        return MH_EINVAL;
    }
    NvtxScope range("mh_step_timesym");
    const double dir = backward ? -1.0 : 1.0;
    const std::pair<int, int> key(n_iter, backward ? 1 : 0);
    int64_t k = 0;
    while (k < nsteps) {
        // Two consecutive steps use the two banks of Eq. 24 words in turn and end
        // where they began (H- in bank 0, word n_iter - 1), so from there pairs of
        // steps replay one captured CUDA graph: the per-launch host cost of small
        // systems goes away.  Plain launches: the first step(s), an odd last
        // step, and while per-launch timing is on.
        const bool graphable = sim->s.ts_prev == n_iter - 1 && nsteps - k >= 2 && !sim->timing &&
                               sim->s.part != nullptr;
        if (!graphable) {
            if (int rc = timesym_step(sim, n_iter, dir)) return rc;
            ++k;
            continue;
        }
        auto it = sim->ts_graphs.find(key);
        if (it == sim->ts_graphs.end()) {
            const mh_counters before = sim->ctr;
            cudaGraph_t g = nullptr;
            MH_CUDA(cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal));
            int rc = timesym_step(sim, n_iter, dir);
            if (!rc) rc = timesym_step(sim, n_iter, dir);
            cudaError_t e = cudaStreamEndCapture(sim->stream, &g);
            mh_counters inc = sim->ctr;
            sim->ctr = before;
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "mh_step_timesym: stream capture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "mh_step_timesym: graph instantiation");
            inc.steps -= before.steps;
            inc.evaluations -= before.evaluations;
            inc.pair_interactions -= before.pair_interactions;
            inc.particle_steps -= before.particle_steps;
            inc.kernel_launches -= before.kernel_launches;
            sim->ts_graph_inc[key] = inc;
            it = sim->ts_graphs.emplace(key, ex).first;
        }
        MH_CUDA(cudaGraphLaunch(it->second, sim->stream));
        const mh_counters &inc = sim->ts_graph_inc[key];
        sim->ctr.steps += inc.steps;
        sim->ctr.evaluations += inc.evaluations;
        sim->ctr.pair_interactions += inc.pair_interactions;
        sim->ctr.particle_steps += inc.particle_steps;
        sim->ctr.kernel_launches += inc.kernel_launches;
        k += 2;
    }
    return MH_OK;
}

int mh_step(mh_sim *sim, double dt, int n_iter)
{
    if (int rc = check_handle(sim)) return rc;
    if (!(dt != 0.0) || !std::isfinite(dt)) { set_error("mh_step: dt must be finite and non-zero"); return MH_EINVAL; }
    if (n_iter < 1 || n_iter > 64) { set_error("mh_step: n_iter must be in [1, 64]"); return MH_EINVAL; }
    if (int rc = injected_step_fault("mh_step")) return rc;
    NvtxScope range("mh_step");
    if (sim->batch) { set_error("mh_step: batched simulations advance with mh_step_batch"); return MH_EINVAL; }
    if (sim->cfg.step_mode == MH_STEP_BLOCK) return block_advance(sim, dt, n_iter);
    if (sim->cfg.step_mode == MH_STEP_TIMESYM) {
        set_error("mh_step: time-symmetric simulations advance with mh_step_timesym");
        return MH_EINVAL;
    }
    return shared_step(sim, dt, n_iter, -1.0, nullptr);
}

static int ensure_conv(mh_sim *sim)
{
    if (sim->conv) return MH_OK;
    MH_CUDA(cudaMalloc((void **)&sim->conv, 2 * sizeof(unsigned long long)));
    MH_CUDA(cudaMallocHost((void **)&sim->conv_host, 2 * sizeof(unsigned long long)));
    return MH_OK;
}

int mh_step_converge(mh_sim *sim, double dt, double tol, int max_iter, int *n_used)
{
    if (int rc = check_handle(sim)) return rc;
    if (!(dt != 0.0) || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1 || max_iter > 64) {
        set_error("mh_step_converge: dt finite and non-zero, tol >= 0, 1 <= max_iter <= 64");
        return MH_EINVAL;
    }
    if (sim->batch || sim->cfg.step_mode != MH_STEP_SHARED) {
        set_error("mh_step_converge: shared-step simulations only");
        return MH_EINVAL;
    }
    if (int rc = ensure_conv(sim)) return rc;
    return shared_step(sim, dt, max_iter, tol, n_used);
}

int mh_set_predictor(mh_sim *sim, mh_mlp *net)
{
    if (int rc = check_handle(sim)) return rc;
    if (sim->batch || sim->cfg.step_mode != MH_STEP_SHARED) {
        set_error("mh_set_predictor: shared-step simulations only");
        return MH_EINVAL;
    }
    if (net) {
        if (sim->s.p > 3) {
            set_error("mh_set_predictor: the learned residual is built for orders 4 to 8");
            return MH_EINVAL;
        }
        int n_in = 0, n_out = 0;
        mlp_dims(net, &n_in, &n_out);
        if (n_in != 6 * sim->s.p + 1 || n_out != 6) {
            set_error("mh_set_predictor: the network must map 6p + 1 features to 6 outputs");
            return MH_EINVAL;
        }
        if (!sim->lfeat) {
            MH_CUDA(cudaMalloc((void **)&sim->lfeat, (size_t)sim->s.N * (6 * sim->s.p + 1) * sizeof(float)));
            MH_CUDA(cudaMalloc((void **)&sim->lout, (size_t)sim->s.N * 6 * sizeof(float)));
        }
    }
    sim->mlp = net;
    return MH_OK;
}

int mh_predict(mh_sim *sim, double dt, double *x, double *v)
{
    if (int rc = check_handle(sim)) return rc;
    if (!x || !v || !(dt != 0.0) || !std::isfinite(dt)) { set_error("mh_predict: host x, v and dt != 0"); return MH_EINVAL; }
    if (sim->batch || sim->cfg.step_mode != MH_STEP_SHARED) { set_error("mh_predict: shared-step simulations only"); return MH_EINVAL; }
    DeviceState &s = sim->s;
    int rc = launch_step_phase(s, sim->cfg, dt, 0, false, 0, sim->stream);
    if (rc) return rc;
    s.flip ^= 1;
    if (sim->mlp) {
        if ((rc = launch_learned_features(s, dt, sim->lfeat, sim->stream))) return rc;
        if ((rc = mlp_infer(sim->mlp, sim->lfeat, sim->lout, s.N, sim->stream))) return rc;
        if ((rc = launch_learned_apply(s, sim->cfg, dt, sim->lout, 1e3f, sim->stream))) return rc;
        s.flip ^= 1;
    }
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    std::vector<double> h(3 * s.Np);
    MH_CUDA(cudaMemcpy(h.data(), s.x1, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost));
    from_soa(h, s.N, 1, s.Np, x);
    MH_CUDA(cudaMemcpy(h.data(), s.v1, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost));
    from_soa(h, s.N, 1, s.Np, v);
    return MH_OK;
}

int mh_collect_samples(mh_sim *sim, double dt, int n_iter, float *feats, float *targets)
{
    if (int rc = check_handle(sim)) return rc;
    if (!feats || !targets || !(dt != 0.0) || !std::isfinite(dt) || n_iter < 1 || n_iter > 64) {
        set_error("mh_collect_samples: device feats/targets, dt != 0, 1 <= n_iter <= 64");
        return MH_EINVAL;
    }
    if (sim->batch || sim->cfg.step_mode != MH_STEP_SHARED || sim->s.p > 3) {
        set_error("mh_collect_samples: shared-step simulations of order 4 to 8 only");
        return MH_EINVAL;
    }
    DeviceState &s = sim->s;
    const size_t K = 2 * s.p;
    if (!sim->lsave) MH_CUDA(cudaMalloc((void **)&sim->lsave, (6 + 3 * K) * s.Np * sizeof(double)));
    double *xs = sim->lsave, *vs = xs + 3 * s.Np, *ds = vs + 3 * s.Np;
    MH_CUDA(cudaMemcpyAsync(xs, s.x0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream));
    MH_CUDA(cudaMemcpyAsync(vs, s.v0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream));
    MH_CUDA(cudaMemcpyAsync(ds, s.d0, 3 * K * s.Np * sizeof(double), cudaMemcpyDeviceToDevice, sim->stream));
    mh_mlp *keep = sim->mlp;
    sim->mlp = nullptr;                 // samples come from the plain predictor and a converged corrector
    int rc = shared_step(sim, dt, n_iter, -1.0, nullptr);
    sim->mlp = keep;
    if (rc) return rc;
    rc = launch_collect(s, dt, xs, vs, ds, feats, targets, sim->stream);
    if (rc) return rc;
    sim->ctr.kernel_launches += 1;
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return MH_OK;
}

static int check_flag(mh_sim *sim)
{
    int flag = 0;
    MH_CUDA(cudaMemcpyAsync(&flag, sim->s.flag, sizeof(int), cudaMemcpyDeviceToHost, sim->stream));
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    if (flag & kFlagSymWait) {
        // the ordered accumulation's counters may be left mid-way: clear them for
        // later launches; the state itself is invalid and stays flagged
        DeviceState &s = sim->s;
        if (s.symsync) MH_CUDA(cudaMemsetAsync(s.symsync, 0, s.symsync_words * sizeof(unsigned), sim->stream));
        MH_CUDA(cudaStreamSynchronize(sim->stream));
        set_error("a pair-symmetric evaluation waited longer than its limit for its turn to add its sums; "
                  "the state is invalid");
        return MH_ETIMEOUT;
    }
    if (flag) {
        set_error("non-finite position or velocity produced by a step");
        return MH_ENONFINITE;
    }
    return MH_OK;
}

int mh_sync(mh_sim *sim, mh_state *out)
{
    if (int rc = check_handle(sim)) return rc;
    if (!out) { set_error("mh_sync: out is NULL"); return MH_EINVAL; }
    if (fault_armed("nonfinite")) {
        set_error("non-finite position or velocity (injected by MH_FAULT=nonfinite)");
        return MH_ENONFINITE;
    }
    DeviceState &s = sim->s;
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    if (int rc = collect_timing(sim)) return rc;
    if (s.tst) MH_CUDA(cudaMemcpy(&sim->t, s.tst, sizeof(double), cudaMemcpyDeviceToHost));
    out->t = sim->t;
    std::vector<double> h;
    if (out->x) {
        h.resize(3 * s.Np);
        MH_CUDA(cudaMemcpy(h.data(), s.x0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost));
        from_soa(h, s.N, 1, s.Np, out->x);
    }
    if (out->v) {
        h.resize(3 * s.Np);
        MH_CUDA(cudaMemcpy(h.data(), s.v0, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost));
        from_soa(h, s.N, 1, s.Np, out->v);
    }
    if (out->derivs) {
        const int K = 2 * s.p;
        h.resize((size_t)K * 3 * s.Np);
        MH_CUDA(cudaMemcpy(h.data(), s.d0, (size_t)K * 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost));
        from_soa(h, s.N, K, s.Np, out->derivs);
    }
    if (out->level && s.level) MH_CUDA(cudaMemcpy(out->level, s.level, s.N * sizeof(int), cudaMemcpyDeviceToHost));
    return check_flag(sim);
}

int mh_set_state(mh_sim *sim, const mh_state *in)
{
    if (int rc = check_handle(sim)) return rc;
    if (sim->batch && !in->derivs) { set_error("mh_set_state: a batched simulation needs derivs"); return MH_EINVAL; }
    if (!in || !in->x || !in->v) { set_error("mh_set_state: x and v are required"); return MH_EINVAL; }
    DeviceState &s = sim->s;
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    std::vector<double> h;
    to_soa(in->x, s.N, 1, s.Np, h, kFarAway);
    MH_CUDA(cudaMemcpy(s.x0, h.data(), 3 * s.Np * sizeof(double), cudaMemcpyHostToDevice));
    to_soa(in->v, s.N, 1, s.Np, h, 0.0);
    MH_CUDA(cudaMemcpy(s.v0, h.data(), 3 * s.Np * sizeof(double), cudaMemcpyHostToDevice));
    MH_CUDA(cudaMemsetAsync(s.flag, 0, sizeof(int), sim->stream));
    if (s.symsync) MH_CUDA(cudaMemsetAsync(s.symsync, 0, s.symsync_words * sizeof(unsigned), sim->stream));
    if (int rc = upload_bounds(s, in->x, in->v, sim->stream)) return rc;
    sim->t = in->t;
    if (s.tst) MH_CUDA(cudaMemcpy(s.tst, &in->t, sizeof(double), cudaMemcpyHostToDevice));
    if (s.comp) MH_CUDA(cudaMemset(s.comp, 0, 6 * s.Np * sizeof(double)));   // a new state starts exact
    if (in->derivs) {
        to_soa(in->derivs, s.N, 2 * s.p, s.Np, h, 0.0);
        MH_CUDA(cudaMemcpy(s.d0, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else if (int rc = initialise(sim)) {
        return rc;
    }
    if (int rc = timesym_start(sim)) return rc;
    if (sim->cfg.step_mode == MH_STEP_BLOCK) {
        // every body restarts at the given time; levels from the caller or the criterion
        s.T_now = 0;
        if (int rc = launch_block_init(s, sim->cfg, sim->stream)) return rc;
        if (in->level) {
            for (int64_t i = 0; i < s.N; ++i)
                if (in->level[i] < 0 || in->level[i] > sim->cfg.k_max) {
                    set_error("mh_set_state: level out of [0, k_max]");
                    return MH_EINVAL;
                }
            MH_CUDA(cudaMemcpyAsync(s.level, in->level, s.N * sizeof(int), cudaMemcpyHostToDevice, sim->stream));
        }
    }
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return MH_OK;
}

int mh_diagnostics(mh_sim *sim, double *energy, double *ecc, int central)
{
    if (int rc = check_handle(sim)) return rc;
    if (sim->batch && energy) { set_error("mh_diagnostics: use mh_batch_energy for batched simulations"); return MH_EINVAL; }
    DeviceState &s = sim->s;
    if (ecc && (central < 0 || central >= s.N)) { set_error("mh_diagnostics: central index out of range"); return MH_EINVAL; }
    double *e_rows = s.diag;
    double *e_scalar = s.diag + 3 * s.Np;
    double *scratch = e_scalar + 1;
    if (energy) {
        if (int rc = launch_energy(s, sim->eps, sim->cfg.G, scratch, e_scalar, sim->stream)) return rc;
        MH_CUDA(cudaMemcpyAsync(energy, e_scalar, sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
        sim->ctr.kernel_launches += 2;
    }
    if (ecc) {
        if (int rc = launch_ecc(s, sim->cfg.G, central, e_rows, sim->stream)) return rc;
        sim->ctr.kernel_launches += 1;
        std::vector<double> h(3 * s.Np);
        MH_CUDA(cudaMemcpyAsync(h.data(), e_rows, 3 * s.Np * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
        MH_CUDA(cudaStreamSynchronize(sim->stream));
        from_soa(h, s.N, 1, s.Np, ecc);
    }
    MH_CUDA(cudaStreamSynchronize(sim->stream));
    return check_flag(sim);
}

int mh_set_timing(mh_sim *sim, int on)
{
    if (int rc = check_handle(sim)) return rc;
    sim->timing = on != 0;
    return MH_OK;
}

int mh_info(mh_sim *sim, int64_t *N, int *order, mh_counters *counters)
{
    if (int rc = check_handle(sim)) return rc;
    if (int rc = collect_timing(sim)) return rc;
    if (N) *N = sim->s.N;
    if (order) *order = sim->cfg.order;
    if (counters) *counters = sim->ctr;
    return MH_OK;
}

}  // extern "C"

// ---- kernel-level entry point on caller-owned device memory ----

namespace {
struct Scratch {
    double *part = nullptr;
    size_t doubles = 0;
    float *rows32 = nullptr;
    size_t floats = 0;
    unsigned long long *bound = nullptr;
    size_t nbound = 0;
};
Scratch g_scratch[64];

template <typename T>
int grow(T **ptr, size_t *cap, size_t need, cudaStream_t st)
{
    if (need <= *cap) return MH_OK;
    MH_CUDA(cudaStreamSynchronize(st));
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    MH_CUDA(cudaMalloc((void **)ptr, need * sizeof(T)));
    *cap = need;
    return MH_OK;
}
}  // namespace

extern "C" {

int mh_pair_eval(int P, int precision, int64_t N, const double *m, const double *traj, double eps,
                 double G, int64_t i0, int64_t i1, double *out, void *stream)
{
    set_error("");
    const bool ok_p = precision == MH_PREC_FP64 ? (P >= 1 && P <= 5)
                    : precision == MH_PREC_FP32PAIR ? (P >= 1 && P <= 3) : false;
    if (!ok_p) {
        set_error("mh_pair_eval: P must be 1..5 (FP64) or 1..3 (FP32-pair)");
        return MH_EINVAL;
    }
    if (N < 1 || !m || !traj || !out || i0 < 0 || i1 > N || i0 >= i1 || !(eps >= 0.0)) {
        set_error("mh_pair_eval: need N >= 1, device pointers, 0 <= i0 < i1 <= N, eps >= 0");
        return MH_EINVAL;
    }
    int dev = 0;
    MH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("mh_pair_eval: device index out of range"); return MH_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n_i = i1 - i0;
    const PairPlan pl = plan_pair(P, precision, n_i, N, 0, dev);
    Scratch &sc = g_scratch[dev];
    int rc = grow(&sc.part, &sc.doubles, (size_t)pl.split * (P + 1) * 3 * n_i, st);
    if (rc) return rc;
    if (precision == MH_PREC_FP32PAIR) {
        if ((rc = grow(&sc.rows32, &sc.floats, (size_t)nf32(P) * N, st))) return rc;
        if ((rc = grow(&sc.bound, &sc.nbound, 2, st))) return rc;
        if ((rc = launch_split32(N, P, traj, m, G, sc.rows32, sc.bound, st))) return rc;
    }
    rc = launch_pair(P, precision, N, N, m, traj, sc.rows32, eps, G, i0, i1, sc.part, n_i, pl, st);
    if (rc) return rc;
    return launch_reduce_out(n_i, n_i, (P + 1) * 3, pl.split, sc.part, out, st);
}

int mh_release_scratch(void)
{
    int dev = 0;
    MH_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) {
        Scratch &sc = g_scratch[dev];
        if (sc.part || sc.rows32 || sc.bound) MH_CUDA(cudaDeviceSynchronize());
        if (sc.part) cudaFree(sc.part);
        if (sc.rows32) cudaFree(sc.rows32);
        if (sc.bound) cudaFree(sc.bound);
        sc = Scratch{};
    }
    return MH_OK;
}

}  // extern "C"
