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

// Merge key of a range lookup: (window start i, slot) from its row index
// r = slot * n + i.  Within one node's list the window starts strictly
// increase (the runs ascend and a run's windows start at a, a + w, ...,
// a + L - w), so every list is sorted by this key.
__device__ __forceinline__ uint64_t lookup_key(uint32_t r, uint32_t n) {
    uint32_t slot = 0;
#pragma unroll
    for (int k = 1; k < kMaxTableRows; k++) slot += (uint64_t)r >= (uint64_t)k * n ? 1u : 0u;
    return ((uint64_t)(r - slot * n) << 3) | slot;
}

// Entries of each list a merging lane loads at a time (independent loads).
constexpr int kMergeWindow = 4;

// First index of list[0 .. len) whose key is >= k (the list is sorted by key).
__device__ __forceinline__ uint32_t key_lower_bound(const uint32_t *__restrict__ list, uint32_t len, uint64_t k,
                                                    uint32_t n) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (lookup_key(list[mid], n) < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per group of up to NODES nodes: merge the group's lookup lists by
// key; equal keys (the same row) become one entry whose class is the set of
// lists holding it.  The key space is split among the lanes at 31 keys
// sampled evenly from the group's longest list, and every lane merges its own
// key range serially.  Without WRITE: count the group's entries of every class
// into cc[group << NODES | class].  With WRITE: from those counts, write the
// group's class descriptors (classes in increasing mask order, empty ones left
// out) and its rows, sorted by class (within a class by key), at rows[b ...].
// Shared memory: 2^NODES counters or write cursors per lane.
template <int NODES, bool WRITE>
__global__ void group_merge_kernel(const GroupItem *__restrict__ items, uint64_t n_groups,
                                   const uint64_t *__restrict__ lk_off, const uint32_t *__restrict__ lk, uint32_t n,
                                   uint32_t *__restrict__ cc, uint32_t *__restrict__ lane_cc,
                                   uint32_t *__restrict__ rows, uint2 *__restrict__ cls) {
    extern __shared__ __align__(16) uint32_t s_cnt[];
    constexpr uint32_t C = 1u << NODES;
    const int lane = threadIdx.x & 31;
    const uint64_t gid = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gid >= n_groups) return;
    uint32_t *c = s_cnt + (threadIdx.x >> 5) * (C * 32) + lane;  // c[k * 32]: this lane's counter of class k

    const GroupItem &it = items[gid];
    const uint32_t *list[NODES];
    uint32_t len[NODES];
    const uint32_t *longest = lk;  // the longest list (not indexed by a run-time subscript)
    uint32_t L = 0;
#pragma unroll
    for (int j = 0; j < NODES; j++) {
        const uint32_t v = it.node[j];
        const uint64_t o = v == 0xffffffffu ? 0 : lk_off[v];
        list[j] = lk + o;
        len[j] = v == 0xffffffffu ? 0u : (uint32_t)(lk_off[v + 1] - o);
        if (len[j] > L) {
            L = len[j];
            longest = list[j];
        }
    }
    // this lane's key range [k0, k1)
    uint64_t k0 = lane == 0 || L == 0 ? 0ull : lookup_key(longest[(uint32_t)((uint64_t)L * lane / 32)], n);
    uint64_t k1 = __shfl_down_sync(0xffffffffu, k0, 1);
    if (lane == 31) k1 = ~0ull;
    uint32_t p[NODES], p0[NODES], e[NODES];
    uint64_t hk[NODES];
    uint32_t win[NODES][kMergeWindow];  // the next entries of each list, loaded together
    auto load_windows = [&]() {
#pragma unroll
        for (int j = 0; j < NODES; j++) {
            p0[j] = p[j];
#pragma unroll
            for (int q = 0; q < kMergeWindow; q++) win[j][q] = p[j] + q < e[j] ? list[j][p[j] + q] : 0u;
            hk[j] = p[j] < e[j] ? lookup_key(win[j][0], n) : ~0ull;
        }
    };
#pragma unroll
    for (int j = 0; j < NODES; j++) {
        p[j] = k0 == 0 ? 0u : key_lower_bound(list[j], len[j], k0, n);
        e[j] = k1 == ~0ull ? len[j] : key_lower_bound(list[j], len[j], k1, n);
    }
    load_windows();
    uint32_t *mine = cc + (gid << NODES);
    for (uint32_t k = 0; k < C; k++) c[k * 32] = 0;
    uint32_t *my_lane_cc = lane_cc ? lane_cc + (gid << NODES) * 32 + lane : nullptr;  // [group][class][lane]
    if (WRITE && my_lane_cc) {
        for (uint32_t k = 0; k < C; k++) c[k * 32] = my_lane_cc[k * 32];
    } else if (WRITE) {
        // this lane's count in every class, found by a merge pass that only
        // counts (when the count pass kept no per-lane counts)
        for (;;) {
            uint64_t best = ~0ull;
#pragma unroll
            for (int j = 0; j < NODES; j++) best = hk[j] < best ? hk[j] : best;
            if (best == ~0ull) break;
            uint32_t mask = 0;
#pragma unroll
            for (int j = 0; j < NODES; j++)
                if (hk[j] == best) {
                    mask |= 1u << j;
                    p[j]++;
                    hk[j] = p[j] < e[j] ? lookup_key(list[j][p[j]], n) : ~0ull;
                }
            c[mask * 32]++;
        }
#pragma unroll
        for (int j = 0; j < NODES; j++) p[j] = k0 == 0 ? 0u : key_lower_bound(list[j], len[j], k0, n);
        load_windows();
    }
    if (WRITE) {
        // this lane's cursor in class k: the class's base (classes in mask
        // order) plus the counts of the lower lanes
        uint32_t base = 0;
        uint64_t ci = it.cls;
        for (uint32_t k = 1; k < C; k++) {
            const uint32_t total = mine[k];
            if (total == 0) continue;  // warp-uniform
            uint32_t mycount = c[k * 32], excl = mycount;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, excl, o);
                if (lane >= o) excl += y;
            }
            c[k * 32] = base + excl - mycount;
            if (lane == 0) cls[ci] = make_uint2(k, total);
            ci++;
            base += total;
        }
    }
    uint32_t *row_base = WRITE ? rows + it.b : nullptr;
    for (;;) {
        uint64_t best = ~0ull;
#pragma unroll
        for (int j = 0; j < NODES; j++) best = hk[j] < best ? hk[j] : best;
        if (best == ~0ull) break;
        uint32_t mask = 0, r = 0;
#pragma unroll
        for (int j = 0; j < NODES; j++)
            if (hk[j] == best) {
                mask |= 1u << j;
                r = win[j][0];
                p[j]++;
                // shift the look-ahead window; refill it with independent loads when empty
#pragma unroll
                for (int q = 0; q < kMergeWindow - 1; q++) win[j][q] = win[j][q + 1];
                if (p[j] < e[j] && ((p[j] - p0[j]) % kMergeWindow) == 0) {
#pragma unroll
                    for (int q = 0; q < kMergeWindow; q++)
                        win[j][q] = p[j] + q < e[j] ? list[j][p[j] + q] : 0u;
                }
                hk[j] = p[j] < e[j] ? lookup_key(win[j][0], n) : ~0ull;
            }
        if (WRITE)
            row_base[c[mask * 32]++] = r;
        else
            c[mask * 32]++;
    }
    if (!WRITE) {
        __syncwarp();
        for (uint32_t k = 0; k < C; k++) {
            const uint32_t t = __reduce_add_sync(0xffffffffu, c[k * 32]);
            if (lane == 0) mine[k] = t;
            if (my_lane_cc) my_lane_cc[k * 32] = c[k * 32];
        }
    }
}

}  // namespace

static uint64_t l2_size(int device) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    return (uint64_t)(l2 > 0 ? l2 : (64 << 20));
}

uint64_t union_l2_budget(int device) { return l2_size(device) * 3 / 4; }

uint64_t grouped_l2_budget(int device) { return l2_size(device) * 5 / 4; }

static std::atomic<uint32_t> g_scheme_nodes{0};  // vga_set_table_scheme_nodes (0 = from the L2 size)

int table_scheme_auto(uint32_t n, int device) {
    const uint32_t above = g_scheme_nodes.load();
    if (above) return n > above - 1u ? 1 : 0;
    return (uint64_t)table_rows(0) * n * 128u > grouped_l2_budget(device) ? 1 : 0;
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

namespace vga {

int ensure_group_list(const vga_graph *g, int scheme, uint32_t hub_lookups, int nodes, cudaStream_t stream,
                      GroupList *out) {
    if (nodes != 2 && nodes != 4 && nodes != 8) {
        set_error("internal: group size %d", nodes);
        return VGA_EINVAL;
    }
    VGA_TRY(ensure_run_lookups(g, scheme, stream));
    std::lock_guard<std::mutex> lock(g->lk_mu);
    if (hub_lookups == 0) hub_lookups = 1;
    vga_graph::RunLookups &L = g->lk[scheme];
    auto publish = [&](const vga_graph::RunLookups::GroupSet &gs) {
        *out = GroupList{static_cast<const GroupItem *>(gs.d_items), gs.count, static_cast<const uint32_t *>(gs.d_rows),
                         static_cast<const uint2 *>(gs.d_cls), gs.rows_used, gs.hub_rows, gs.nodes};
    };
    for (const vga_graph::RunLookups::GroupSet &gs : L.groups)
        if (gs.hub_lookups == hub_lookups && gs.nodes == nodes) {
            publish(gs);
            return VGA_OK;
        }
    // groups of consecutive non-hub nodes; a group closes early rather than
    // hold 2^31 or more lookups (its merged count stays a u32)
    const std::vector<uint64_t> &off = L.h_off;
    std::vector<GroupItem> items;
    GroupItem cur{};
    int k = 0;
    uint64_t sum = 0, hub_rows = 0;
    auto close = [&]() {
        for (int j = k; j < kGroupMaxNodes; j++) cur.node[j] = 0xffffffffu;
        items.push_back(cur);
        cur = GroupItem{};
        k = 0;
        sum = 0;
    };
    auto add = [&](uint32_t v) {
        const uint64_t cnt = off[v + 1] - off[v];
        if (cnt > hub_lookups) {  // split hubs stay per node
            hub_rows += cnt;
            return;
        }
        if (k && sum + cnt >= (1ull << 31)) close();
        cur.node[k++] = v;
        sum += cnt;
    };
    if (!g->cells.empty() && g->cells.size() == g->n) {
        // with the grid geometry: blocks of cells (2 x 1, 2 x 2 or 4 x 2), in
        // raster order of blocks, each block's nodes in raster order
        const int W = g->cells_W, H = g->cells_H;
        const int bw = nodes == 2 ? 2 : nodes == 4 ? 2 : 4, bh = nodes == 2 ? 1 : 2;
        std::vector<uint32_t> node_of((size_t)W * H, 0xffffffffu);
        for (uint32_t v = 0; v < g->n; v++) node_of[g->cells[v]] = v;
        for (int by = 0; by < H; by += bh)
            for (int bx = 0; bx < W; bx += bw) {
                for (int dy = 0; dy < bh && by + dy < H; dy++)
                    for (int dx = 0; dx < bw && bx + dx < W; dx++) {
                        const uint32_t v = node_of[(size_t)(by + dy) * W + bx + dx];
                        if (v != 0xffffffffu) add(v);
                    }
                if (k) close();
            }
    } else {
        // consecutive ids
        for (uint32_t v = 0; v < g->n; v++) {
            add(v);
            if (k == nodes) close();
        }
        if (k) close();
    }
    const uint64_t ng = items.size();
    const int warps = nodes >= 8 ? 1 : 4;  // one warp per group; 32 lanes x 2^nodes counters each
    const size_t smem = (size_t)warps * 32 * (4u << nodes);
    DeviceBuffer d_items, d_cc, d_lane_cc;
    VGA_TRY(d_items.alloc(sizeof(GroupItem) * std::max<uint64_t>(ng, 1)));
    VGA_TRY(d_cc.alloc((4ull << nodes) * std::max<uint64_t>(ng, 1)));
    // per-lane class counts of the count pass, which spare the write pass a
    // recount (groups of up to 4 nodes: 2 KB a group)
    if (nodes <= 4) VGA_TRY(d_lane_cc.alloc((128ull << nodes) * std::max<uint64_t>(ng, 1)));
    auto merge = [&](bool write, uint32_t *rows, uint2 *cls) -> int {
        if (!ng) return VGA_OK;
        VGA_CHECK_CUDA(cudaMemcpyAsync(d_items.ptr, items.data(), sizeof(GroupItem) * ng, cudaMemcpyHostToDevice,
                                       stream));
        const unsigned blocks = (unsigned)((ng + warps - 1) / warps);
        const int threads = warps * 32;
#define VGA_GM(NN)                                                                                                   \
    if (write)                                                                                                       \
        group_merge_kernel<NN, true><<<blocks, threads, smem, stream>>>(d_items.as<GroupItem>(), ng, L.d_off,       \
                                                                        L.d_lk, g->n, d_cc.as<uint32_t>(),           \
                                                                        d_lane_cc.as<uint32_t>(), rows, cls);        \
    else                                                                                                             \
        group_merge_kernel<NN, false><<<blocks, threads, smem, stream>>>(d_items.as<GroupItem>(), ng, L.d_off,      \
                                                                         L.d_lk, g->n, d_cc.as<uint32_t>(),          \
                                                                         d_lane_cc.as<uint32_t>(), rows, cls)
        if (nodes == 2) VGA_GM(2);
        else if (nodes == 4) VGA_GM(4);
        else {
            static std::once_flag once;
            static cudaError_t attr = cudaSuccess;
            std::call_once(once, [] {
                attr = cudaFuncSetAttribute(group_merge_kernel<8, false>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * 256 * 4);
                if (attr == cudaSuccess)
                    attr = cudaFuncSetAttribute(group_merge_kernel<8, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * 256 * 4);
            });
            VGA_CHECK_CUDA(attr);
            VGA_GM(8);
        }
#undef VGA_GM
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        return VGA_OK;
    };
    VGA_TRY(merge(false, nullptr, nullptr));
    std::vector<uint32_t> h_cc((size_t)ng << nodes);
    if (ng) VGA_CHECK_CUDA(cudaMemcpyAsync(h_cc.data(), d_cc.ptr, 4 * h_cc.size(), cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    uint64_t rows_total = 0, rows_used = 0, cls_total = 0;
    for (uint64_t i = 0; i < ng; i++) {
        uint64_t r = 0;
        uint32_t nc = 0;
        for (uint32_t m = 1; m < (1u << nodes); m++) {
            r += h_cc[(i << nodes) + m];
            nc += h_cc[(i << nodes) + m] ? 1u : 0u;
        }
        items[i].b = rows_total;
        items[i].cnt = (uint32_t)r;
        items[i].nc = nc;
        items[i].cls = cls_total;
        rows_total += (r + 3) & ~3ull;  // each group's rows start on a 16-byte boundary (TMA)
        rows_used += r;
        cls_total += nc;
    }
    DeviceBuffer d_rows, d_cls;
    VGA_TRY(d_rows.alloc(4 * (rows_total + 4)));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_rows.ptr, 0, 4 * (rows_total + 4), stream));
    VGA_TRY(d_cls.alloc(sizeof(uint2) * std::max<uint64_t>(cls_total, 1)));
    VGA_TRY(merge(true, d_rows.as<uint32_t>(), d_cls.as<uint2>()));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));  // the host vectors go out of scope
    L.groups.push_back(vga_graph::RunLookups::GroupSet{hub_lookups, nodes, ng, rows_total, rows_used, hub_rows,
                                                       d_items.release(), d_rows.release(), d_cls.release()});
    publish(L.groups.back());
    return VGA_OK;
}

}  // namespace vga
