// noalloc.cu -- gift_filter_noalloc: the filter with no device allocation.
//
// Some callers cannot allocate device memory while they filter: code that
// runs under a fixed memory budget set aside in advance, real-time loops
// where an allocation's latency or a failure mid-loop is not acceptable, or
// hosts that hand this library device buffers but own the allocator.  For
// them the filter's scratch (intermediate signals, accumulator, scale
// vectors) lives in one file-scope device array of fixed size, held by every
// GPU that loads it until the process exits.
//
// With lazy module loading the array is only reserved when its module is
// first loaded on a device, which the address lookup below triggers.
// gift_ctx_create does that lookup (noalloc_reserve), so the reservation, and
// any failure to make it, happens when a context is created and never inside
// a gift_filter_noalloc call.
#include <map>
#include <mutex>

#include "internal.cuh"

namespace gift {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GIFT_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array for the current device, looked up
// once per device (the array's name in host code is only a stand-in).
void *scratch_address(int device) {
    static std::mutex mu;
    static std::map<int, void *> addr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = addr.find(device);
    if (it != addr.end()) return it->second;
    void *p = nullptr;
    GIFT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[device] = p;
    return p;
}

}  // namespace

void noalloc_reserve(int device) { (void)scratch_address(device); }

}  // namespace gift

using namespace gift;

extern "C" gift_status gift_filter_noalloc(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec,
                                           const float *g_in, int32_t num_signals, float *g_out, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_filter_noalloc: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        gift_filter_spec def;
        if (!spec) {
            gift_filter_spec_default(&def);
            spec = &def;
        }
        GIFT_REQUIRE(num_signals >= 1, "gift_filter_noalloc: num_signals must be >= 1");
        // the size estimate walks spec->term[0 .. num_terms): check the count first
        GIFT_REQUIRE(spec->num_terms >= 1 && spec->num_terms <= GIFT_MAX_TERMS,
                     "gift_filter_noalloc: num_terms out of range");
        const size_t need = filter_scratch_bytes(graph, spec, num_signals);
        if (need > (size_t)GIFT_NOALLOC_SCRATCH_BYTES)
            throw Failure{GIFT_ERR_INVALID, "gift_filter_noalloc: needs " + std::to_string(need) +
                                                " bytes of scratch, more than the fixed " +
                                                std::to_string((size_t)GIFT_NOALLOC_SCRATCH_BYTES) + " bytes"};
        void *scratch = scratch_address(ctx->device);
        filter_on_scratch(ctx, graph, spec, g_in, num_signals, g_out, scratch, (size_t)GIFT_NOALLOC_SCRATCH_BYTES,
                          static_cast<cudaStream_t>(stream));
    });
}
