// run.cu -- the whole path in one call from host memory (gift_run): the
// signal's upload runs on a side stream while the graph is built on the
// caller's stream; the filter waits for it, HPWL follows on the device, and
// the result comes back in one copy.
#include <cstring>

#include "internal.cuh"

using namespace gift;

extern "C" gift_status gift_run(gift_ctx *ctx, const gift_netlist *netlist, const gift_build_opts *opts,
                                const gift_filter_spec *spec, const float *g_in, int32_t num_signals, float *g_out,
                                double *hpwl, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && netlist, "gift_run: NULL context or netlist");
        GIFT_REQUIRE(netlist->mem == GIFT_MEM_HOST, "gift_run: the netlist must be in host memory");
        GIFT_REQUIRE(g_in && g_out, "gift_run: NULL signal pointer");
        GIFT_REQUIRE(num_signals >= 1, "gift_run: num_signals must be >= 1");
        GIFT_REQUIRE(netlist->num_cells > 0, "gift_run: num_cells must be > 0");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        gift_filter_spec def;
        if (!spec) {
            gift_filter_spec_default(&def);
            spec = &def;
        }
        {
            std::lock_guard<std::mutex> lk(ctx->side_mu);
            if (!ctx->side) GIFT_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        }
        const size_t bytes = sizeof(float) * (size_t)netlist->num_cells * 2 * num_signals;
        DevBuf din(ctx, bytes, st), dout(ctx, bytes, st), bad(ctx, sizeof(int32_t), st);
        GIFT_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), st));
        cudaEvent_t ready = nullptr, loaded = nullptr;
        GIFT_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        struct Events {
            cudaEvent_t &a, &b;
            ~Events() {
                if (a) cudaEventDestroy(a);
                if (b) cudaEventDestroy(b);
            }
        } own{ready, loaded};
        GIFT_CUDA(cudaEventCreateWithFlags(&loaded, cudaEventDisableTiming));
        // g goes up on the side stream behind the netlist's copies (so the
        // two do not share the link while the build waits for the netlist),
        // overlapping the build's kernels
        bool queued = false;
        auto upload = [&] {
            GIFT_CUDA(cudaEventRecord(ready, st));
            std::lock_guard<std::mutex> lk(ctx->side_mu);
            GIFT_CUDA(cudaStreamWaitEvent(ctx->side, ready, 0));
            GIFT_CUDA(cudaMemcpyAsync(din.p, g_in, bytes, cudaMemcpyHostToDevice, ctx->side));
            scan_nonfinite(ctx, din.as<float>(), (int64_t)netlist->num_cells * 2 * num_signals, bad.as<int32_t>(),
                           ctx->side);
            GIFT_CUDA(cudaEventRecord(loaded, ctx->side));
            queued = true;
        };
        // on every way out (an invalid netlist throws from the build), the
        // stream waits for the side stream's copies before din and dout are
        // freed on it
        struct WaitSide {
            cudaStream_t st;
            cudaEvent_t &ev;
            const bool &armed;
            ~WaitSide() {
                if (armed) cudaStreamWaitEvent(st, ev, 0);
            }
        } wait_side{st, loaded, queued};
        gift_graph *g = nullptr;
        build_graph_impl(ctx, netlist, opts, &g, st, upload);
        struct Graph {
            gift_graph *g;
            cudaStream_t st;
            ~Graph() {
                release_graph(g, st);
                cudaStreamSynchronize(st);
                delete g;
            }
        } gown{g, st};
        if (!queued) upload();
        // a signal with a NaN or an infinity is rejected before the filter runs
        GIFT_CUDA(cudaStreamWaitEvent(st, loaded, 0));
        int32_t hbad = 0;
        GIFT_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        GIFT_REQUIRE(!hbad, "gift_run: g_in holds a NaN or an infinity");
        // g_out in page-locked host memory: the last sweep stores the result
        // there as it goes; otherwise it goes down on the side stream while
        // HPWL reads the device copy on st
        float *mirror = host_mirror(g_out, bytes);
        filter_impl(ctx, g, spec, din.as<float>(), num_signals, dout.as<float>(), GIFT_MEM_DEVICE, st, mirror);
        if (!mirror) {
            GIFT_CUDA(cudaEventRecord(ready, st));
            std::lock_guard<std::mutex> lk(ctx->side_mu);
            GIFT_CUDA(cudaStreamWaitEvent(ctx->side, ready, 0));
            GIFT_CUDA(cudaMemcpyAsync(g_out, dout.p, bytes, cudaMemcpyDeviceToHost, ctx->side));
            GIFT_CUDA(cudaEventRecord(loaded, ctx->side));
        }
        if (hpwl) hpwl_impl(ctx, g, dout.as<float>(), num_signals, hpwl, GIFT_MEM_DEVICE, st);
        GIFT_CUDA(cudaEventSynchronize(loaded));
        sync_and_check(ctx, st);
    });
}
