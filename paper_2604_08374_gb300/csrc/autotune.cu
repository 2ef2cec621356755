// autotune.cu -- per-degree-bucket choice of the union's launch shape.
//
// The union (Eq. hll-union) computes the same registers under every launch
// choice: the variant (one gather per neighbour, or per run of consecutive
// ids), the slice width S, the CTA size and the hub threshold only change how
// fast.  Which is fastest depends mostly on the degree: it sets how long a
// node's list is, how many runs it breaks into, and how far one warp's work
// spreads.  The tuner groups graphs by floor(log2(E/N)), times the candidates
// on the bucket's largest graph and keeps the fastest; the table it fills is
// consulted by every analysis whose tuning fields are left at 0.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "vga_common.cuh"

namespace vga {
namespace {

std::mutex g_tab_mu;
std::vector<vga_tune_entry> g_tab;

int degree_bucket(const vga_graph *g) {
    if (!g || g->n == 0 || g->n_edges == 0) return -1;
    const uint64_t avg = g->n_edges / g->n;
    return avg ? 63 - __builtin_clzll(avg) : 0;
}

bool entry_ok(const vga_tune_entry &e) {
    return (e.union_mode == 1 || e.union_mode == 2) && e.slice_bytes >= 16 && e.slice_bytes <= 1024 &&
           !(e.slice_bytes & (e.slice_bytes - 1)) && e.warps_per_cta >= 0 && e.warps_per_cta <= 16 &&
           e.hub_lookups >= 0 &&
           (e.group_nodes == 0 || e.group_nodes == 1 || e.group_nodes == 2 || e.group_nodes == 4 ||
            e.group_nodes == 8);
}

// Union time of two passes (d = 2), the faster of two runs; < 0 on failure.
int time_candidate(const vga_graph *g, int p, const vga_tuning &t, cudaStream_t stream, double *ms) {
    double best = -1.0;
    for (int rep = 0; rep < 2; rep++) {
        double u = 0.0;
        int it = 0;
        VGA_TRY(run_timed(g, p, 2, 0x5eedull, &t, stream, &u, &it));
        if (u > 0.0 && (best < 0.0 || u < best)) best = u;
    }
    *ms = best;
    return VGA_OK;
}

int tune_graph(const vga_graph *g, int p, cudaStream_t stream, vga_tune_entry *e) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device);
    const uint64_t l2_bytes = (uint64_t)(l2 > 0 ? l2 : (64 << 20));
    const uint32_t m = 1u << p;
    vga_tuning best{};
    double best_ms = -1.0;
    auto consider = [&](const vga_tuning &t) -> int {
        double ms = -1.0;
        VGA_TRY(time_candidate(g, p, t, stream, &ms));
        if (ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) {
            best_ms = ms;
            best = t;
        }
        return VGA_OK;
    };
    // 1. variant x slice width, 8 warps, automatic hub threshold
    for (int mode = 1; mode <= 2; mode++) {
        if (mode == 2 && (uint64_t)g->n > kRunMaxNodes) continue;
        const uint64_t rows = mode == 2 ? (uint64_t)table_rows(g->lk_scheme) : 1;
        for (uint32_t S = 16; S <= std::min<uint32_t>(m, 1024u); S <<= 1) {
            if (S > 16 && (uint64_t)S * g->n * rows > l2_bytes) break;
            vga_tuning t{};
            t.union_mode = mode;
            t.slice_bytes = (int)S;
            t.warps_per_cta = 8;
            VGA_TRY(consider(t));
        }
    }
    if (best_ms < 0.0) {
        set_error("vga_autotune: no candidate could be timed");
        return VGA_ECUDA;
    }
    // 2. CTA size
    const vga_tuning base = best;
    for (int w : {4, 16}) {
        vga_tuning t = base;
        t.warps_per_cta = w;
        VGA_TRY(consider(t));
    }
    // 3. hub threshold (mode 2): the automatic one, then smaller
    if (best.union_mode == 2) {
        const uint32_t autoh = hub_lookups_auto(g, g->lk_scheme);
        const vga_tuning base2 = best;
        for (uint32_t div : {2u, 4u}) {
            vga_tuning t = base2;
            t.hub_lookups = (int)std::max<uint32_t>(autoh / div, 64u);
            VGA_TRY(consider(t));
        }
    }
    // 4. group size of the grouped union (mode 2): one node per warp, 2 and 8
    //    against the automatic 4
    if (best.union_mode == 2) {
        const vga_tuning base3 = best;
        for (int gn : {1, 2, 8}) {
            vga_tuning t = base3;
            t.group_nodes = gn;
            VGA_TRY(consider(t));
        }
    }
    e->degree_log2 = degree_bucket(g);
    e->group_nodes = best.group_nodes;
    e->union_mode = best.union_mode;
    e->slice_bytes = best.slice_bytes;
    e->warps_per_cta = best.warps_per_cta;
    e->hub_lookups = best.hub_lookups;
    e->p = p;
    e->geu_per_s = 2.0 * (double)g->n_edges / (best_ms * 1e-3) / 1e9;
    e->tuned_edges = g->n_edges;
    return VGA_OK;
}

}  // namespace

bool tune_table_lookup(const vga_graph *g, vga_tune_entry *out) {
    const int b = degree_bucket(g);
    if (b < 0) return false;
    std::lock_guard<std::mutex> lock(g_tab_mu);
    for (const vga_tune_entry &e : g_tab)
        if (e.degree_log2 == b) {
            *out = e;
            return true;
        }
    return false;
}

}  // namespace vga

using namespace vga;

extern "C" {

int vga_tune_table_set(const vga_tune_entry *entries, int n) {
    clear_error();
    if (n < 0 || (n > 0 && !entries)) {
        set_error("vga_tune_table_set: bad entry list");
        return VGA_EINVAL;
    }
    for (int i = 0; i < n; i++)
        if (!entry_ok(entries[i])) {
            set_error("vga_tune_table_set: entry %d has union_mode %d, slice_bytes %d, warps_per_cta %d, "
                      "hub_lookups %d, group_nodes %d",
                      i, entries[i].union_mode, entries[i].slice_bytes, entries[i].warps_per_cta,
                      entries[i].hub_lookups, entries[i].group_nodes);
            return VGA_EINVAL;
        }
    std::lock_guard<std::mutex> lock(g_tab_mu);
    g_tab.assign(entries, entries + n);
    return VGA_OK;
}

int vga_tune_table_get(vga_tune_entry *out, int max_out, int *n_out) {
    clear_error();
    if (!n_out || max_out < 0 || (max_out > 0 && !out)) {
        set_error("vga_tune_table_get: bad output arguments");
        return VGA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_tab_mu);
    const int n = (int)std::min<size_t>(g_tab.size(), (size_t)max_out);
    std::copy(g_tab.begin(), g_tab.begin() + n, out);
    *n_out = (int)g_tab.size();
    return VGA_OK;
}

int vga_autotune(const vga_graph *const *graphs, int n_graphs, int p, void *stream_ptr, vga_tune_entry *out,
                 int max_out, int *n_out, int install) {
    clear_error();
    if (!graphs || n_graphs < 1 || !out || !n_out || max_out < 1 || p < 4 || p > 16) {
        set_error("vga_autotune: need graphs, n_graphs >= 1, an output array and 4 <= p <= 16");
        return VGA_EINVAL;
    }
    int dev = -1;
    VGA_CHECK_CUDA(cudaGetDevice(&dev));
    // the largest graph of each bucket
    std::vector<const vga_graph *> rep(64, nullptr);
    for (int i = 0; i < n_graphs; i++) {
        const vga_graph *g = graphs[i];
        if (!g) {
            set_error("vga_autotune: graph %d is null", i);
            return VGA_EINVAL;
        }
        if (g->device != dev) {
            set_error("vga_autotune: graph %d lives on device %d, device %d is current", i, g->device, dev);
            return VGA_EINVAL;
        }
        const int b = degree_bucket(g);
        if (b < 0) continue;
        if (!rep[b] || g->n_edges > rep[b]->n_edges) rep[b] = g;
    }
    int count = 0;
    for (const vga_graph *g : rep) count += g != nullptr;
    if (count > max_out) {
        set_error("vga_autotune: %d degree buckets present, room for %d", count, max_out);
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    // tune without the installed table steering the candidates' untouched fields
    std::vector<vga_tune_entry> saved;
    {
        std::lock_guard<std::mutex> lock(g_tab_mu);
        saved.swap(g_tab);
    }
    int k = 0, rc = VGA_OK;
    for (const vga_graph *g : rep) {
        if (!g) continue;
        rc = tune_graph(g, p, stream, &out[k]);
        if (rc != VGA_OK) break;
        k++;
    }
    {
        std::lock_guard<std::mutex> lock(g_tab_mu);
        if (rc == VGA_OK && install)
            g_tab.assign(out, out + k);
        else
            g_tab.swap(saved);
    }
    *n_out = k;
    return rc;
}

}  // extern "C"
