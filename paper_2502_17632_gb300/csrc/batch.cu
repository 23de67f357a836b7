// batch.cu -- many netlists filtered together, and filters replayed as CUDA
// graphs.
//
// A batch of B netlists becomes one block-diagonal graph: graph b's cells,
// nets and pins follow those of graphs 0..b-1 (ids offset), so no edge joins
// two graphs and each row holds exactly the nonzeros, weights (same nets, same
// net order, same FP64 sums) and degree it has when its graph is built alone.
// One gift_filter over the batch therefore runs every graph's filter in the
// same launches (one pass per sweep over all B graphs), with per-graph
// results bit-identical to filtering each graph alone with the same kernel
// shape.  gift_hpwl_batch gives each graph's HPWL.
//
// gift_filter_capture records one filter call -- every sweep, scale and
// packing kernel -- as a CUDA graph on scratch memory the handle owns, so a
// batch is filtered by a single graph launch.
#include <algorithm>
#include <cstring>
#include <memory>

#include "internal.cuh"

namespace gift {
namespace {

// dst[i] = src[i] + add for i < n; flags a source value outside [0, limit).
__global__ void k_offset_i64(int64_t n, const int64_t *__restrict__ src, int64_t add, int64_t *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}
__global__ void k_offset_i32(int64_t n, const int32_t *__restrict__ src, int32_t add, int32_t limit,
                             int32_t *__restrict__ dst, int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = src[i];
        if (v < 0 || v >= limit) *bad = 1;
        dst[i] = v + add;
    }
}

int grid_of(gift_ctx *ctx, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 8));
}

}  // namespace
}  // namespace gift

using namespace gift;

struct gift_exec {
    gift_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *scratch = nullptr;
};

extern "C" {

gift_status gift_build_batch(gift_ctx *ctx, const gift_netlist *nets, int32_t B, const gift_build_opts *opts,
                             gift_graph **out, int64_t *cell_offsets, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && nets && out, "gift_build_batch: NULL argument");
        GIFT_REQUIRE(B >= 1, "gift_build_batch: num_graphs must be >= 1");
        *out = nullptr;
        GIFT_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int32_t mem = nets[0].mem;
        GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_build_batch: bad mem kind");
        std::vector<int64_t> cells(B + 1, 0), nts(B + 1, 0), pins(B + 1, 0);
        std::vector<int64_t> ends(2 * (size_t)B, 0);
        for (int b = 0; b < B; ++b) {
            const gift_netlist &nl = nets[b];
            GIFT_REQUIRE(nl.mem == mem, "gift_build_batch: every netlist must be in the same memory kind");
            GIFT_REQUIRE(nl.num_cells > 0 && nl.num_nets >= 0, "gift_build_batch: bad netlist sizes");
            GIFT_REQUIRE(nl.net_ptr != nullptr, "gift_build_batch: net_ptr is NULL");
            if (mem == GIFT_MEM_HOST) {
                ends[2 * b] = nl.net_ptr[0];
                ends[2 * b + 1] = nl.net_ptr[nl.num_nets];
            } else {
                GIFT_CUDA(cudaMemcpyAsync(&ends[2 * b], nl.net_ptr, 8, cudaMemcpyDeviceToHost, st));
                GIFT_CUDA(cudaMemcpyAsync(&ends[2 * b + 1], nl.net_ptr + nl.num_nets, 8, cudaMemcpyDeviceToHost, st));
            }
        }
        if (mem == GIFT_MEM_DEVICE) GIFT_CUDA(cudaStreamSynchronize(st));
        for (int b = 0; b < B; ++b) {
            GIFT_REQUIRE(ends[2 * b] == 0 && ends[2 * b + 1] >= 0, "gift_build_batch: net_ptr must start at 0");
            GIFT_REQUIRE(ends[2 * b + 1] == 0 || nets[b].pin_cell, "gift_build_batch: pin_cell is NULL");
            cells[b + 1] = cells[b] + nets[b].num_cells;
            nts[b + 1] = nts[b] + nets[b].num_nets;
            pins[b + 1] = pins[b] + ends[2 * b + 1];
        }
        GIFT_REQUIRE(cells[B] < ((int64_t)1 << 31) - 1 && nts[B] < ((int64_t)1 << 31) - 1,
                     "gift_build_batch: the batch has too many cells or nets");
        const int64_t N = cells[B], E = nts[B], P = pins[B];
        gift_netlist cat;
        cat.num_cells = (int32_t)N;
        cat.num_nets = (int32_t)E;
        cat.mem = mem;
        std::vector<int64_t> hnp;
        std::vector<int32_t> hpc;
        std::vector<uint8_t> hfx;
        DevBuf dnp, dpc, dfx, dbad;
        if (mem == GIFT_MEM_HOST) {
            hnp.resize(E + 1);
            hpc.resize(std::max<int64_t>(P, 1));
            hfx.assign(N, 0);
            for (int b = 0; b < B; ++b) {
                const gift_netlist &nl = nets[b];
                for (int32_t e = 0; e < nl.num_nets; ++e) hnp[nts[b] + e] = nl.net_ptr[e] + pins[b];
                for (int64_t q = 0; q < ends[2 * b + 1]; ++q) {
                    const int32_t c = nl.pin_cell[q];
                    GIFT_REQUIRE(c >= 0 && c < nl.num_cells, "gift_build_batch: pin cell out of range");
                    hpc[pins[b] + q] = c + (int32_t)cells[b];
                }
                if (nl.is_fixed) std::memcpy(hfx.data() + cells[b], nl.is_fixed, nl.num_cells);
            }
            hnp[E] = P;
            cat.net_ptr = hnp.data();
            cat.pin_cell = hpc.data();
            cat.is_fixed = hfx.data();
        } else {
            dnp = DevBuf(ctx, sizeof(int64_t) * (E + 1), st);
            dpc = DevBuf(ctx, sizeof(int32_t) * std::max<int64_t>(P, 1), st);
            dfx = DevBuf(ctx, N, st);
            dbad = DevBuf(ctx, sizeof(int), st);
            GIFT_CUDA(cudaMemsetAsync(dbad.p, 0, sizeof(int), st));
            for (int b = 0; b < B; ++b) {
                const gift_netlist &nl = nets[b];
                if (nl.num_nets > 0)
                    k_offset_i64<<<grid_of(ctx, nl.num_nets), 256, 0, st>>>(nl.num_nets, nl.net_ptr, pins[b],
                                                                           dnp.as<int64_t>() + nts[b]);
                const int64_t pb = ends[2 * b + 1];
                if (pb > 0)
                    k_offset_i32<<<grid_of(ctx, pb), 256, 0, st>>>(pb, nl.pin_cell, (int32_t)cells[b], nl.num_cells,
                                                                 dpc.as<int32_t>() + pins[b], dbad.as<int>());
                if (nl.is_fixed)
                    GIFT_CUDA(cudaMemcpyAsync(dfx.as<uint8_t>() + cells[b], nl.is_fixed, nl.num_cells,
                                              cudaMemcpyDeviceToDevice, st));
                else
                    GIFT_CUDA(cudaMemsetAsync(dfx.as<uint8_t>() + cells[b], 0, nl.num_cells, st));
            }
            check_launch("k_offset");
            GIFT_CUDA(cudaMemcpyAsync(dnp.as<int64_t>() + E, &P, sizeof(int64_t), cudaMemcpyHostToDevice, st));
            int bad = 0;
            GIFT_CUDA(cudaMemcpyAsync(&bad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            GIFT_REQUIRE(bad == 0, "gift_build_batch: pin cell out of range");
            cat.net_ptr = dnp.as<int64_t>();
            cat.pin_cell = dpc.as<int32_t>();
            cat.is_fixed = dfx.as<uint8_t>();
        }
        gift_graph *g = nullptr;
        build_graph_impl(ctx, &cat, opts, &g, st);
        g->seg_cells = cells;
        g->seg_nets = nts;
        if (cell_offsets) std::copy(cells.begin(), cells.end(), cell_offsets);
        *out = g;
    });
}

gift_status gift_hpwl_batch(gift_ctx *ctx, const gift_graph *graph, const float *xy, int32_t num_signals,
                            double *out, int32_t mem, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_hpwl_batch: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        hpwl_batch_impl(ctx, graph, xy, num_signals, out, mem, static_cast<cudaStream_t>(stream));
    });
}

gift_status gift_filter_capture(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec,
                                const float *g_in, int32_t num_signals, float *g_out, gift_exec **out) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph && out, "gift_filter_capture: NULL argument");
        *out = nullptr;
        GIFT_CUDA(cudaSetDevice(ctx->device));
        gift_filter_spec def;
        if (!spec) {
            gift_filter_spec_default(&def);
            spec = &def;
        }
        cudaStream_t cs;
        GIFT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        auto ex = std::make_unique<gift_exec>();
        ex->ctx = ctx;
        try {
            // one ordinary call first: tunes the shapes and builds the formats
            // they use, so the captured call allocates nothing and never waits
            filter_impl(ctx, graph, spec, g_in, num_signals, g_out, GIFT_MEM_DEVICE, cs);
            const size_t bytes = filter_scratch_bytes(graph, spec, num_signals);
            GIFT_CUDA(cudaMalloc(&ex->scratch, bytes));
            GIFT_CUDA(cudaStreamSynchronize(cs));
            {
                TimerPause pause;  // no timing events inside the capture
                GIFT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                try {
                    filter_on_scratch(ctx, graph, spec, g_in, num_signals, g_out, ex->scratch, bytes, cs);
                } catch (...) {
                    cudaGraph_t broken = nullptr;
                    cudaStreamEndCapture(cs, &broken);
                    if (broken) cudaGraphDestroy(broken);
                    throw;
                }
                GIFT_CUDA(cudaStreamEndCapture(cs, &ex->graph));
            }
            GIFT_CUDA(cudaGraphInstantiate(&ex->exec, ex->graph, 0));
        } catch (...) {
            if (ex->exec) cudaGraphExecDestroy(ex->exec);
            if (ex->graph) cudaGraphDestroy(ex->graph);
            if (ex->scratch) cudaFree(ex->scratch);
            cudaStreamDestroy(cs);
            throw;
        }
        cudaStreamDestroy(cs);
        *out = ex.release();
    });
}

gift_status gift_exec_launch(gift_exec *ex, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ex != nullptr, "gift_exec_launch: NULL handle");
        GIFT_CUDA(cudaSetDevice(ex->ctx->device));
        GIFT_CUDA(cudaGraphLaunch(ex->exec, static_cast<cudaStream_t>(stream)));
    });
}

void gift_exec_free(gift_exec *ex) {
    if (!ex) return;
    cudaSetDevice(ex->ctx->device);
    cudaDeviceSynchronize();
    if (ex->exec) cudaGraphExecDestroy(ex->exec);
    if (ex->graph) cudaGraphDestroy(ex->graph);
    if (ex->scratch) cudaFree(ex->scratch);
    delete ex;
}

}  // extern "C"
