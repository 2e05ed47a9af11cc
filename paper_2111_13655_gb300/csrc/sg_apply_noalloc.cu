// sg_apply_H_noalloc: y = H_S x with the apply's scratch memory taken from a
// fixed array compiled into this library instead of device memory allocated
// at run time.
//
// Who needs this: a caller that may not call cudaMalloc at the point where it
// applies H.  Examples are a host program whose device memory has been handed
// in full to another allocator (a framework's caching pool that reserved the
// GPU up front, so a fresh cudaMalloc would fail or fragment it), and a
// latency-critical loop that cannot take the implicit device-wide
// synchronisation a cudaMalloc/cudaFree may cause.  sg_apply_H allocates its
// fixed-point accumulators on the first call with a larger nvec; this entry
// point never allocates.
//
// The scratch holds, per call, the per-vector scale exponents (kNoAllocMaxVec
// words) followed by the fixed-point accumulators of the compact vectors
// (sg::acc_words words per element: four for FP64 contexts, one for mixed).  It is one array shared by every call on a
// device, and keeps whatever the last call left in it: each call clears the
// part it uses before its kernels run.  Two calls whose GPU work overlaps
// (different streams, host threads or contexts on the same device) use the
// same words and race; the caller must order them.
#include <mutex>
#include <string>

#include "sg_internal.h"

namespace {

// 16 MiB: kNoAllocMaxVec exponent words + (16 MiB / 8 - 64) = 2,097,088 words
// of accumulators: 524,272 vector elements (nvec * N_cs) for FP64 contexts,
// 2,097,088 for mixed-precision contexts.
constexpr size_t kNoAllocWords = (size_t)SG_NOALLOC_SCRATCH_BYTES / sizeof(unsigned long long);
constexpr int kNoAllocMaxVec = SG_NOALLOC_MAX_NVEC;
constexpr size_t kNoAllocAccWords = kNoAllocWords - kNoAllocMaxVec;
static_assert(SG_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");
static_assert(kNoAllocAccWords / sg::acc_words(false) == SG_NOALLOC_MAX_ELEMS, "header limit out of date");
static_assert(kNoAllocAccWords / sg::acc_words(true) == SG_NOALLOC_MAX_ELEMS_MIXED, "header limit out of date");

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

// Device address of g_noalloc_scratch per device ordinal.  Host code may not
// use the symbol itself as a pointer (it names a host-side shadow), so the
// address is asked from the runtime once per device, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
unsigned long long *g_addr[kMaxDevices] = {};

sg_status noalloc_fail(sg_ctx *ctx, sg_status st, const std::string &msg)
{
    ctx->last_error = "sg_apply_H_noalloc: " + msg;
    return st;
}

}  // namespace

extern "C" sg_status sg_apply_H_noalloc(sg_ctx *ctx, const double *x, double *y, int nvec, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) return noalloc_fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return noalloc_fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    if (!x || !y) return noalloc_fail(ctx, SG_EINVAL, "x or y is NULL");
    if (nvec < 1) return noalloc_fail(ctx, SG_EINVAL, "nvec must be >= 1");
    const size_t n = (size_t)ctx->host.n_cs * (size_t)nvec;
    const size_t words = (size_t)sg::acc_words(ctx->fp32);
    const size_t max_elems = kNoAllocAccWords / words;
    if (nvec > kNoAllocMaxVec || n > max_elems)
        return noalloc_fail(ctx, SG_EUNSUPPORTED,
                            "nvec * N_cs = " + std::to_string(n) + " with nvec = " + std::to_string(nvec) +
                                " exceeds the fixed scratch (nvec <= " + std::to_string(kNoAllocMaxVec) +
                                ", nvec * N_cs <= " + std::to_string(max_elems) +
                                (ctx->fp32 ? " for mixed-precision contexts" : " for FP64 contexts") +
                                "); use sg_apply_H");
    if ((x < y + n) && (y < x + n)) return noalloc_fail(ctx, SG_EINVAL, "x and y overlap");

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(ctx, SG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != ctx->device)
        return noalloc_fail(ctx, SG_EINVAL, "the context's device (" + std::to_string(ctx->device) +
                                                ") is not the current device (" + std::to_string(dev) + ")");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(ctx, SG_EUNSUPPORTED, "device ordinal >= 64");

    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_addr_mutex);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return noalloc_fail(ctx, SG_ECUDA,
                                    std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = static_cast<unsigned long long *>(p);
        }
        scratch = g_addr[dev];
    }

    cudaStream_t s = (cudaStream_t)stream;
    long long *maxbits = reinterpret_cast<long long *>(scratch);
    unsigned long long *acc = scratch + kNoAllocMaxVec;
    // The accumulators are summed into and must start at zero; the exponents
    // are cleared by the launch itself.
    e = cudaMemsetAsync(acc, 0, n * words * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return noalloc_fail(ctx, SG_ECUDA, std::string("memset: ") + cudaGetErrorString(e));

    sg::KParams kp = ctx->kp;
    kp.acc = acc;
    kp.xs = nullptr;  // no staged input copy: the term kernels read x
    e = sg::launch_apply(kp, ctx->fp32, x, y, nvec, maxbits, nullptr, s);
    if (e != cudaSuccess) return noalloc_fail(ctx, SG_ECUDA, std::string("apply launch: ") + cudaGetErrorString(e));
    return SG_OK;
}
