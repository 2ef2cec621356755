// runs.cu -- range lookups for the run-aware union.
//
// Eq. hll-union takes the register-wise max over a node's neighbours.  In a
// visibility graph numbered in raster order (Sec. 3.2) a neighbour list is a
// sequence of runs of consecutive ids: a visible stretch of a grid row is a
// block of consecutive node ids (the paper's one-byte deltas of 1).  On the
// 236k-cell city graph a list of ~20k neighbours has ~1.8k runs.  The max over
// a run [a, a+L) equals the max of two overlapping power-of-two windows of a
// sparse table T_k[i] = max(cur[i .. i + 2^k)), so each run costs one or two
// gathers instead of L; runs of 32 or more are covered by ceil(L/16) windows of
// 16.  Max is associative, commutative and idempotent, so the result is the
// same register array, bit for bit.
//
// This file turns the LEB128 CSR into the list of lookups of every node, once
// per graph: one warp per node decodes its list with the warp window decoder,
// finds run boundaries across windows, and emits each completed run's lookups
// as row indices k * N + i of a slice's table region (T_0 = the slice, then
// T_1..T_4), so that the union addresses a row with one multiply-add.
#include <algorithm>
#include <vector>

#include "runs.cuh"

namespace vga {
namespace {

// One warp per node: write node v's lookups at lk[lk_off[v] ...] (their
// counts were taken when the graph was validated).
__global__ void run_lookups_kernel(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes, uint32_t n,
                                   const uint64_t *__restrict__ lk_off, uint32_t *__restrict__ lk) {
    __shared__ uint32_t s_ids[8][128];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *ids = s_ids[wib];
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n) return;
    const uint32_t v = (uint32_t)warp;
    uint64_t pos = off[v];
    const uint64_t end = off[v + 1];
    uint32_t base = 0;
    RunTracker rt;
    rt.out = lk_off[v];
    while (pos < end) {
        int advance = 0;
        uint32_t next = 0;
        bool unused = false;
        const int c = decode_window4<uint32_t, false>(bytes, pos, end, base, lane, ids, advance, next, false, 0, 0,
                                                      unused);
        if (c == 0) break;  // cannot happen on a validated graph
        __syncwarp();
        rt.window<true>(ids, c, lane, n, lk);
        __syncwarp();
        base = next;
        pos += (uint64_t)advance;
    }
    rt.finish<true>(lane, n, lk);
}

}  // namespace

int ensure_run_lookups(const vga_graph *g, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g->lk_mu);
    if (g->lk_ready) return VGA_OK;
    if ((uint64_t)g->n > kRunMaxNodes) {
        set_error("run-aware union supports at most 2^29 nodes (graph has %u)", g->n);
        return VGA_EINVAL;
    }
    const uint32_t n = g->n;
    const std::vector<uint64_t> &h_off = g->h_lk_off;  // prefix sums of the counts taken at load
    const uint64_t total = h_off[n];
    DeviceBuffer d_off, d_lk;
    VGA_TRY(d_off.alloc(8 * ((size_t)n + 1)));
    VGA_TRY(d_lk.alloc(4 * ((size_t)total + 4)));  // + one 16-byte group: TMA copies round up to whole groups
    VGA_CHECK_CUDA(cudaMemsetAsync(d_lk.as<uint8_t>() + 4 * total, 0, 16, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_off.ptr, h_off.data(), 8 * ((size_t)n + 1), cudaMemcpyHostToDevice, stream));
    if (n) {
        const int warps = 8;
        const unsigned blocks = (unsigned)(((uint64_t)n + warps - 1) / warps);
        run_lookups_kernel<<<blocks, warps * 32, 0, stream>>>(g->d_offsets, g->d_bytes, n, d_off.as<uint64_t>(),
                                                              d_lk.as<uint32_t>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    g->d_lk_off = static_cast<uint64_t *>(d_off.release());
    g->d_lk = static_cast<uint32_t *>(d_lk.release());
    g->lk_total = total;
    g->lk_ready = true;
    return VGA_OK;
}

uint32_t hub_lookups_auto(const vga_graph *g) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const uint64_t share = g->lk_total / ((uint64_t)(sms > 0 ? sms : 1) * 64);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(share / 2, 2048), 0x7fffffffull);
}

int ensure_run_items(const vga_graph *g, uint32_t hub_lookups, cudaStream_t stream, RunItemList *out) {
    VGA_TRY(ensure_run_lookups(g, stream));
    std::lock_guard<std::mutex> lock(g->lk_mu);
    if (hub_lookups == 0) hub_lookups = 1;
    for (const vga_graph::RunItemSet &r : g->lk_items)
        if (r.hub_lookups == hub_lookups) {
            *out = RunItemList{static_cast<const RunItem *>(r.d_items), r.count, r.hub_items, r.hubs};
            return VGA_OK;
        }
    const std::vector<uint64_t> &off = g->h_lk_off;
    std::vector<RunItem> items;
    items.reserve((size_t)g->n);
    uint32_t hubs = 0;
    for (uint32_t v = 0; v < g->n; v++) {
        const uint64_t cnt = off[v + 1] - off[v];
        if (cnt <= hub_lookups) continue;
        const uint64_t k = (cnt + hub_lookups - 1) / hub_lookups;  // chunks of at most hub_lookups
        for (uint64_t c = 0; c < k; c++) {
            const uint64_t lo = off[v] + cnt * c / k, hi = off[v] + cnt * (c + 1) / k;
            items.push_back(RunItem{v | kHubChunk, (uint32_t)(hi - lo), lo});
        }
        hubs++;
    }
    const uint64_t hub_items = items.size();
    for (uint32_t v = 0; v < g->n; v++) {
        const uint64_t cnt = off[v + 1] - off[v];
        if (cnt <= hub_lookups) items.push_back(RunItem{v, (uint32_t)cnt, off[v]});
    }
    DeviceBuffer d;
    VGA_TRY(d.alloc(sizeof(RunItem) * (items.empty() ? 1 : items.size())));
    if (!items.empty())
        VGA_CHECK_CUDA(cudaMemcpyAsync(d.ptr, items.data(), sizeof(RunItem) * items.size(), cudaMemcpyHostToDevice,
                                       stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));  // the host vector goes out of scope
    g->lk_items.push_back(vga_graph::RunItemSet{hub_lookups, (uint64_t)items.size(), hub_items, hubs, d.release()});
    const vga_graph::RunItemSet &r = g->lk_items.back();
    *out = RunItemList{static_cast<const RunItem *>(r.d_items), r.count, r.hub_items, r.hubs};
    return VGA_OK;
}

}  // namespace vga
