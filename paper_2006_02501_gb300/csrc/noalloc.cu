// mh_pair_eval_noalloc: the direct-summation evaluation of mh_pair_eval with
// every byte of scratch taken from one fixed array compiled into the library,
// for callers that must not allocate device memory.
//
// Scratch: g_noalloc_scratch below, kNoAllocBytes bytes per device.  It holds
// the split-j partial sums and, in the precision form, the FP32 hi/lo input
// rows and their two grid bounds.  Every GPU that loads the library holds the
// array until the process exits.
#include <mutex>

#include "common.cuh"

namespace mh {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;     // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, resolved once per device.  In host code
// the symbol itself is only a host-side handle, never a device address.
void *g_scratch_ptr[64] = {nullptr};
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace mh

using namespace mh;

extern "C" int mh_pair_eval_noalloc(int P, int precision, int64_t N, const double *m,
                                    const double *traj, double eps, double G, int64_t i0,
                                    int64_t i1, double *out, void *stream)
{
    set_error("");
    const bool ok_p = precision == MH_PREC_FP64 ? (P >= 1 && P <= 5)
                    : precision == MH_PREC_FP32PAIR ? (P >= 1 && P <= 3) : false;
    if (!ok_p) {
        set_error("mh_pair_eval_noalloc: P must be 1..5 (FP64) or 1..3 (FP32-pair)");
        return MH_EINVAL;
    }
    if (N < 1 || !m || !traj || !out || i0 < 0 || i1 > N || i0 >= i1 || !(eps >= 0.0)) {
        set_error("mh_pair_eval_noalloc: need N >= 1, device pointers, 0 <= i0 < i1 <= N, eps >= 0");
        return MH_EINVAL;
    }
    const int64_t n_i = i1 - i0;
    const size_t rows_bytes = precision == MH_PREC_FP32PAIR ? align256((size_t)nf32(P) * N * sizeof(float)) : 0;
    const size_t bound_bytes = precision == MH_PREC_FP32PAIR ? 256 : 0;
    const size_t slot_bytes = (size_t)(P + 1) * 3 * n_i * sizeof(double);   // one split-j slot
    if (rows_bytes + bound_bytes + align256(slot_bytes) > kNoAllocBytes) {
        set_error("mh_pair_eval_noalloc: problem too large for the fixed 32 MiB scratch (needs " +
                  std::to_string(rows_bytes + bound_bytes + align256(slot_bytes)) +
                  " bytes at the smallest split); use mh_pair_eval");
        return MH_EINVAL;
    }
    int dev = 0;
    MH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("mh_pair_eval_noalloc: device index out of range"); return MH_EINVAL; }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "mh_pair_eval_noalloc: cudaGetSymbolAddress");
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the normal work plan, with the j-split reduced until the partial sums fit
    PairPlan pl = plan_pair(P, precision, n_i, N, 0, dev);
    const size_t avail = kNoAllocBytes - rows_bytes - bound_bytes;
    int split = pl.split;
    while (split > 1 && align256((size_t)split * slot_bytes) > avail) --split;
    if (split != pl.split) pl = plan_pair(P, precision, n_i, N, split, dev);
    const size_t part_bytes = align256((size_t)pl.split * slot_bytes);
    if (part_bytes > avail) {
        set_error("mh_pair_eval_noalloc: internal plan does not fit the scratch");
        return MH_EINVAL;
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    double *part = reinterpret_cast<double *>(b);      // [split][(P+1)*3][n_i]
    float *rows32 = nullptr;
    unsigned long long *bound = nullptr;
    if (precision == MH_PREC_FP32PAIR) {
        rows32 = reinterpret_cast<float *>(b + part_bytes);
        bound = reinterpret_cast<unsigned long long *>(b + part_bytes + rows_bytes);
        // the previous call's contents stay in the array: launch_split32 zeroes
        // the two bounds before raising them
        if (int rc = launch_split32(N, P, traj, m, G, rows32, bound, st)) return rc;
    }
    // every partial-sum entry the reduction reads is written by the evaluation
    if (int rc = launch_pair(P, precision, N, N, m, traj, rows32, eps, G, i0, i1, part, n_i, pl, st))
        return rc;
    return launch_reduce_out(n_i, n_i, (P + 1) * 3, pl.split, part, out, st);
}
