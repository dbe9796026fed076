// Refinement of a selection without any device allocation.
//
// Some callers cannot allocate device memory at the moment they refine: a
// render or UI callback of an interactive view (the brushing of Sec. 5.1.1
// runs there) that must not stall on cudaMalloc, which can synchronise the
// whole device, or a host program whose device memory budget is fixed up
// front and owned by another component. This variant of atsne_refine_subset
// takes its temporary rows from one file-scope device array instead of a
// caller workspace. The array is created when the library is loaded on a
// device and stays allocated on every GPU that loads the library until the
// process exits.
//
// Set-up: the first call on a device, with that device current, resolves the
// array's device address and that of the library's device status word with
// cudaGetSymbolAddress (every first call does, whatever its size, even an
// empty selection). Make that first call before opening any stream capture.
// Later calls on the device reuse the addresses.
//
// Sharing: every call uses the same array, which keeps the previous call's
// contents. Each call writes every temporary value before reading it, so
// nothing needs clearing. Two calls whose work can overlap on the GPU (for
// example on two streams without ordering between them) race on the array:
// order them on one stream or with events.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int64_t NA_ROWS = ATSNE_REFINE_NOALLOC_MAX_ROWS;
constexpr int64_t NA_K = ATSNE_REFINE_NOALLOC_MAX_K;
constexpr size_t NA_SLAB = (size_t)NA_ROWS * NA_K * 4;                 // one [rows][k] 4-byte array
constexpr size_t NA_BYTES = 3 * NA_SLAB + (size_t)NA_ROWS * 4;         // idx, d2, P rows + beta

// The no-allocation scratch: 3 MiB + 8 KiB per device.
static __device__ __align__(256) unsigned char g_refine_scratch[NA_BYTES];

std::mutex g_na_mu;
unsigned char *g_na_ptr[64];

atsne_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "refine_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(ATSNE_EUNSUPPORTED, "refine_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_refine_scratch);
        if (e != cudaSuccess) return cuda_error(e, "refine_noalloc: cudaGetSymbolAddress");
        // the status word the checks below raise is resolved in the same
        // set-up, so no later call needs a symbol lookup
        if (!device_status_word()) return set_error(ATSNE_ECUDA, "refine_noalloc: device status word");
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return ATSNE_OK;
}

}  // namespace
}  // namespace atsne

using namespace atsne;

extern "C" atsne_status atsne_refine_subset_noalloc(const float *X, int64_t N, int32_t D,
                                                    const int32_t *subset, int64_t S, int32_t k,
                                                    float perplexity, int32_t *idx, float *d2,
                                                    float *P_cond, float *beta, float *rho,
                                                    void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!X) return set_error(ATSNE_EINVAL, "X is NULL");
    if (N < 2 || N > INT32_MAX) return set_error(ATSNE_EINVAL, "N=%lld not in [2, 2^31-1]", (long long)N);
    if (D < 1) return set_error(ATSNE_EINVAL, "D=%d < 1", D);
    if (k < 1 || (int64_t)k > N - 1) return set_error(ATSNE_EINVAL, "k=%d not in [1, N-1]", k);
    if (!subset || !idx || !d2 || !P_cond) return set_error(ATSNE_EINVAL, "refine_noalloc: NULL pointer");
    if (S < 0) return set_error(ATSNE_EINVAL, "refine_noalloc: S=%lld < 0", (long long)S);
    if (!(perplexity > 0.f) || !(perplexity < (float)k))
        return set_error(ATSNE_EINVAL, "refine_noalloc: perplexity=%g not in (0, k=%d)", (double)perplexity, k);
    if (S > NA_ROWS)
        return set_error(ATSNE_ENOMEM,
                         "refine_noalloc: %lld rows exceed the fixed scratch of %lld rows; "
                         "use atsne_refine_subset with a workspace",
                         (long long)S, (long long)NA_ROWS);
    if (k > NA_K)
        return set_error(ATSNE_ENOMEM, "refine_noalloc: k=%d exceeds the fixed scratch's k of %lld", k,
                         (long long)NA_K);
    unsigned char *base = nullptr;
    ATSNE_TRY(noalloc_scratch(&base));
    if (S == 0) return ATSNE_OK;
    int32_t *ti = reinterpret_cast<int32_t *>(base);
    float *td = reinterpret_cast<float *>(base + NA_SLAB);
    float *tp = reinterpret_cast<float *>(base + 2 * NA_SLAB);
    float *tb = reinterpret_cast<float *>(base + 3 * NA_SLAB);
    ATSNE_TRY(check_finite(X, N * (int64_t)D, stream));
    ATSNE_TRY(check_indices(subset, S, N, stream));
    ATSNE_TRY(knn_bruteforce(X, N, D, subset, S, k, ti, td, stream));
    ATSNE_TRY(calibrate_launch(td, S, k, perplexity, 1e-5f, 200, tp, tb, stream));
    return refine_scatter_launch(subset, S, N, k, ti, td, tp, tb, idx, d2, P_cond, beta, rho, stream);
}
