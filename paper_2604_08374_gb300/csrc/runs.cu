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
#include <vector>

#include "vga_common.cuh"

namespace vga {
namespace {

// Number of lookups covering the run [a, a + L).
__device__ __forceinline__ uint32_t run_lookup_count(uint32_t L) {
    if (L < 32u) {
        const uint32_t k = 31u - __clz(L);
        return (L == (1u << k)) ? 1u : 2u;
    }
    return (L >> 4) + ((L & 15u) ? 1u : 0u);
}

// Lookups covering the run [a, a + L) as table row indices k * n + i.
__device__ __forceinline__ void run_lookup_write(uint32_t a, uint32_t L, uint32_t n, uint32_t *out) {
    if (L < 32u) {
        const uint32_t k = 31u - __clz(L);
        out[0] = k * n + a;
        if (L != (1u << k)) out[1] = k * n + (a + L - (1u << k));
        return;
    }
    const uint32_t full = L >> 4;
    for (uint32_t j = 0; j < full; j++) out[j] = 4u * n + (a + 16u * j);
    if (L & 15u) out[full] = 4u * n + (a + L - 16u);
}

// One warp per node.  WRITE = false stores the node's lookup count in cnt[v];
// WRITE = true writes the lookups at lk[lk_off[v] ...].
template <bool WRITE>
__global__ void run_lookups_kernel(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes, uint32_t n,
                                   uint64_t *__restrict__ cnt, const uint64_t *__restrict__ lk_off,
                                   uint32_t *__restrict__ lk) {
    __shared__ uint32_t s_ids[8][33];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *ids = s_ids[wib];
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n) return;
    const uint32_t v = (uint32_t)warp;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t pos = off[v];
    const uint64_t end = off[v + 1];
    uint32_t base = 0;
    uint32_t run_a = 0, run_len = 0;  // the run still open at the end of the last window
    uint64_t out = WRITE ? lk_off[v] : 0;
    while (pos < end) {
        const WindowDecode<uint32_t> r = decode_window<uint32_t>(bytes, pos, end, base, lane);
        const uint32_t T = r.term_mask;
        if (T == 0) break;  // cannot happen on a validated graph
        if ((T >> lane) & 1u) ids[__popc(T & lt_mask)] = r.id;
        __syncwarp();
        const int c = __popc(T);
        const uint32_t id = lane < c ? ids[lane] : 0u;
        bool start = false;
        if (lane < c) start = (lane == 0) ? !(run_len > 0 && id == run_a + run_len) : (id != ids[lane - 1] + 1u);
        const uint32_t starts = __ballot_sync(0xffffffffu, start);
        // 1. the open run absorbs the lanes before the window's first start (all
        //    of them if there is none); it is complete once a start follows
        if (run_len > 0) {
            if (starts) {
                run_len += (uint32_t)(__ffs(starts) - 1);
                if (WRITE && lane == 0) run_lookup_write(run_a, run_len, n, lk + out);
                out += run_lookup_count(run_len);
                run_len = 0;
            } else {
                run_len += (uint32_t)c;
            }
        }
        // 2. runs starting in this window: complete if another start follows
        const uint32_t later = starts & ~((2u << lane) - 1u);  // starts after this lane (lane < 31)
        const bool complete = start && lane < 31 && later != 0u;
        const uint32_t L = complete ? (uint32_t)(__ffs(later) - 1 - lane) : 0u;
        const uint32_t my = complete ? run_lookup_count(L) : 0u;
        uint32_t incl = my;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (WRITE && complete) run_lookup_write(id, L, n, lk + out + (incl - my));
        out += __shfl_sync(0xffffffffu, incl, 31);
        // 3. the last start of the window opens a run that may continue
        if (starts) {
            const int last = 31 - __clz(starts);
            run_a = __shfl_sync(0xffffffffu, id, last);
            run_len = (uint32_t)(c - last);
        }
        __syncwarp();
        base = r.next_base;
        pos += (uint64_t)r.advance;
    }
    if (run_len > 0) {
        if (WRITE && lane == 0) run_lookup_write(run_a, run_len, n, lk + out);
        out += run_lookup_count(run_len);
    }
    if (!WRITE && lane == 0) cnt[v] = out;
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
    DeviceBuffer d_cnt, d_off, d_lk;
    VGA_TRY(d_cnt.alloc(8 * (size_t)(n ? n : 1)));
    VGA_TRY(d_off.alloc(8 * ((size_t)n + 1)));
    const int warps = 8;
    const unsigned blocks = (unsigned)(((uint64_t)n + warps - 1) / warps);
    std::vector<uint64_t> h_off((size_t)n + 1, 0);
    if (n) {
        run_lookups_kernel<false><<<blocks, warps * 32, 0, stream>>>(g->d_offsets, g->d_bytes, n,
                                                                     d_cnt.as<uint64_t>(), nullptr, nullptr);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        std::vector<uint64_t> h_cnt(n);
        VGA_CHECK_CUDA(cudaMemcpyAsync(h_cnt.data(), d_cnt.ptr, 8 * (size_t)n, cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        for (uint32_t v = 0; v < n; v++) h_off[v + 1] = h_off[v] + h_cnt[v];
    }
    const uint64_t total = h_off[n];
    VGA_TRY(d_lk.alloc(4 * ((size_t)total + 4)));  // + one 16-byte group: TMA copies round up to whole groups
    VGA_CHECK_CUDA(cudaMemsetAsync(d_lk.as<uint8_t>() + 4 * total, 0, 16, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_off.ptr, h_off.data(), 8 * ((size_t)n + 1), cudaMemcpyHostToDevice, stream));
    if (n) {
        run_lookups_kernel<true><<<blocks, warps * 32, 0, stream>>>(g->d_offsets, g->d_bytes, n, nullptr,
                                                                    d_off.as<uint64_t>(), d_lk.as<uint32_t>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    g->d_lk_off = static_cast<uint64_t *>(d_off.release());
    g->d_lk = static_cast<uint32_t *>(d_lk.release());
    g->lk_total = total;
    g->h_lk_off = std::move(h_off);
    g->lk_ready = true;
    return VGA_OK;
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
