// runs.cu -- range lookups for the run-aware union.
//
// Eq. hll-union takes the register-wise max over a node's neighbours.  In a
// visibility graph numbered in raster order (Sec. 3.2) a neighbour list is a
// sequence of runs of consecutive ids: a visible stretch of a grid row is a
// block of consecutive node ids (the paper's one-byte deltas of 1).  On the
// 236k-cell city graph a list of ~20k neighbours has ~1.8k runs.  The max over
// a run [a, a+L) equals the max of a few overlapping windows of a table of
// range maxima T_k[i] = max(cur[i .. i + 2^k)) (runs.cuh: the widest kept
// width w <= L, ceil(L / w) windows), so each run costs one or a few gathers
// instead of L.  Max is associative, commutative and idempotent, so the
// result is the same register array, bit for bit.
//
// This file turns the LEB128 CSR into the list of lookups of every node, once
// per graph and table scheme: one warp per node walks its list 128 bytes at a
// time, finds the run starts from byte masks (only their varints are
// assembled), and emits each completed run's lookups as row indices slot * N
// + i of a slice's table region, so that the union addresses a row with one
// multiply-add.
#include <algorithm>
#include <atomic>
#include <vector>

#include "runs.cuh"

namespace vga {
namespace {

// One warp per node.  WRITE: write node v's lookups for table scheme `scheme`
// at lk[lk_off[v] ...] (SwarRuns, 128 bytes per step) and check that their
// number is the one counted at validation (*bad = 1 otherwise); without WRITE,
// store their number in cnt[v] (the scheme chosen for the graph is counted by
// validation at load instead).
template <bool WRITE>
__global__ void run_lookups_kernel(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes, uint32_t n,
                                   int scheme, const uint64_t *__restrict__ lk_off, uint32_t *__restrict__ lk,
                                   uint32_t *__restrict__ cnt, int *__restrict__ bad) {
    __shared__ uint32_t s_runs[8][3 * SwarRuns::kRunsCap];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n) return;
    const uint32_t v = (uint32_t)warp;
    const uint64_t pos = off[v], end = off[v + 1];
    SwarRuns r;
    r.scheme = scheme;
    r.out = WRITE ? lk_off[v] : 0;
    for (uint64_t w0 = pos & ~3ull; w0 < end; w0 += 128)
        r.window<WRITE>(bytes, w0, pos, end, lane, n, lk, s_runs[wib]);
    r.finish<WRITE>(lane, n, lk);
    if (lane == 0) {
        if (WRITE && r.out != lk_off[v + 1]) atomicExch(bad, 1);
        if (!WRITE) cnt[v] = (uint32_t)r.out;
    }
}

}  // namespace

uint64_t union_l2_budget(int device) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    return (uint64_t)(l2 > 0 ? l2 : (64 << 20)) * 3 / 4;
}

static std::atomic<uint32_t> g_scheme_nodes{0};  // vga_set_table_scheme_nodes (0 = from the L2 size)

int table_scheme_auto(uint32_t n, int device) {
    const uint32_t above = g_scheme_nodes.load();
    if (above) return n > above - 1u ? 1 : 0;
    return (uint64_t)table_rows(0) * n * 128u > union_l2_budget(device) ? 1 : 0;
}

}  // namespace vga

extern "C" int vga_set_table_scheme_nodes(uint32_t nodes) {
    vga::clear_error();
    vga::g_scheme_nodes.store(nodes);
    return VGA_OK;
}

namespace vga {

int ensure_run_lookups(const vga_graph *g, int scheme, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g->lk_mu);
    if (scheme < 0 || scheme >= kTableSchemes) {
        set_error("internal: table scheme %d", scheme);
        return VGA_EINVAL;
    }
    vga_graph::RunLookups &L = g->lk[scheme];
    if (L.ready) return VGA_OK;
    if ((uint64_t)g->n > kRunMaxNodes) {
        set_error("run-aware union supports at most 2^29 nodes (graph has %u)", g->n);
        return VGA_EINVAL;
    }
    const uint32_t n = g->n;
    const int warps = 8;
    const unsigned blocks = (unsigned)(((uint64_t)n + warps - 1) / warps);
    if (L.h_off.empty()) {  // a scheme other than the one counted at load
        std::vector<uint32_t> h_cnt(n);
        L.h_off.assign((size_t)n + 1, 0);
        if (n) {
            DeviceBuffer d_cnt;
            VGA_TRY(d_cnt.alloc(4 * (size_t)n));
            run_lookups_kernel<false><<<blocks, warps * 32, 0, stream>>>(g->d_offsets, g->d_bytes, n, scheme, nullptr,
                                                                         nullptr, d_cnt.as<uint32_t>(), nullptr);
            count_launch();
            VGA_CHECK_CUDA(cudaGetLastError());
            VGA_CHECK_CUDA(cudaMemcpyAsync(h_cnt.data(), d_cnt.ptr, 4 * (size_t)n, cudaMemcpyDeviceToHost, stream));
            VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        }
        for (uint32_t v = 0; v < n; v++) L.h_off[v + 1] = L.h_off[v] + h_cnt[v];
        L.total = L.h_off[n];
    }
    const uint64_t total = L.total;
    DeviceBuffer d_off, d_lk, d_bad;
    VGA_TRY(d_bad.alloc(4));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_bad.ptr, 0, 4, stream));
    VGA_TRY(d_off.alloc(8 * ((size_t)n + 1)));
    VGA_TRY(d_lk.alloc(4 * ((size_t)total + 4)));  // + one 16-byte group: TMA copies round up to whole groups
    VGA_CHECK_CUDA(cudaMemsetAsync(d_lk.as<uint8_t>() + 4 * total, 0, 16, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_off.ptr, L.h_off.data(), 8 * ((size_t)n + 1), cudaMemcpyHostToDevice, stream));
    if (n) {
        run_lookups_kernel<true><<<blocks, warps * 32, 0, stream>>>(g->d_offsets, g->d_bytes, n, scheme,
                                                                    d_off.as<uint64_t>(), d_lk.as<uint32_t>(),
                                                                    nullptr, d_bad.as<int>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    int bad = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(&bad, d_bad.ptr, 4, cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (bad) {
        set_error("internal: the lookup write pass disagrees with the lookup counts of scheme %d", scheme);
        return VGA_ECORRUPT;
    }
    L.d_off = static_cast<uint64_t *>(d_off.release());
    L.d_lk = static_cast<uint32_t *>(d_lk.release());
    L.ready = true;
    return VGA_OK;
}

uint32_t hub_lookups_auto(const vga_graph *g, int scheme) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const uint64_t share = g->lk[scheme].total / ((uint64_t)(sms > 0 ? sms : 1) * 64);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(share / 2, 2048), 0x7fffffffull);
}

int ensure_run_items(const vga_graph *g, int scheme, uint32_t hub_lookups, cudaStream_t stream, RunItemList *out) {
    VGA_TRY(ensure_run_lookups(g, scheme, stream));
    std::lock_guard<std::mutex> lock(g->lk_mu);
    if (hub_lookups == 0) hub_lookups = 1;
    vga_graph::RunLookups &L = g->lk[scheme];
    for (const vga_graph::RunItemSet &r : L.items)
        if (r.hub_lookups == hub_lookups) {
            *out = RunItemList{static_cast<const RunItem *>(r.d_items), r.count, r.hub_items, r.hubs};
            return VGA_OK;
        }
    const std::vector<uint64_t> &off = L.h_off;
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
    L.items.push_back(vga_graph::RunItemSet{hub_lookups, (uint64_t)items.size(), hub_items, hubs, d.release()});
    const vga_graph::RunItemSet &r = L.items.back();
    *out = RunItemList{static_cast<const RunItem *>(r.d_items), r.count, r.hub_items, r.hubs};
    return VGA_OK;
}

}  // namespace vga
