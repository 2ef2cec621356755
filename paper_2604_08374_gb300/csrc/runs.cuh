// runs.cuh -- run tracking for the run-aware union's range lookups (see
// runs.cu): shared by graph validation, which counts every node's lookups in
// its decode pass, and the pass that writes them.
#pragma once

#include "vga_common.cuh"

namespace vga {
namespace {

// Window width w and region slot of the lookups covering a run of length L:
// the widest kept window not longer than the run (scheme 0: 2^floor(log2 L)
// up to 16; scheme 1: 1, 4 or 16).  ceil(L / w) windows cover it, the last
// one ending at the run's end.
__device__ __forceinline__ void run_window(uint32_t L, int scheme, uint32_t &w, uint32_t &slot) {
    if (scheme == 0) {
        const uint32_t k = L < 16u ? 31u - __clz(L) : 4u;
        w = 1u << k;
        slot = k;
    } else {
        slot = L < 4u ? 0u : (L < 16u ? 1u : 2u);
        w = 1u << (2u * slot);
    }
}

// Number of lookups covering the run [a, a + L).
__device__ __forceinline__ uint32_t run_lookup_count(uint32_t L, int scheme) {
    uint32_t w, slot;
    run_window(L, scheme, w, slot);
    return (L + w - 1u) / w;
}

// Lookups covering the run [a, a + L) as table row indices slot * n + i.
__device__ __forceinline__ void run_lookup_write(uint32_t a, uint32_t L, uint32_t n, int scheme, uint32_t *out) {
    uint32_t w, slot;
    run_window(L, scheme, w, slot);
    const uint32_t c = (L + w - 1u) / w;
    const uint32_t base = slot * n + a;
    for (uint32_t j = 0; j + 1u < c; j++) out[j] = base + w * j;
    out[c - 1u] = base + L - w;
}

// Runs of consecutive ids across a node's decoded windows.  Per window the
// warp passes the window's ids in order in ids[0 .. c), c <= 128; lane L looks
// at ids 4L .. 4L+3.  A run starts at an id that does not follow the one
// before it; a run is complete once the next start is seen (in this window or
// a later one).  `out` counts the lookups emitted so far (WRITE: written at
// lk + out, in order of the runs).
struct RunTracker {
    uint32_t run_a = 0, run_len = 0;  // the run still open at the end of the last window
    uint64_t out = 0;

    int scheme = 0;  // table scheme of the lookups

    template <bool WRITE>
    __device__ __forceinline__ void window(const uint32_t *ids, int c, int lane, uint32_t n, uint32_t *lk) {
        constexpr int kNone = 0x7fffffff;
        const int j0 = 4 * lane;
        uint32_t id[4];
        uint32_t smask = 0;  // run starts among this lane's ids
        uint32_t prev = (j0 > 0 && j0 <= c) ? ids[j0 - 1] : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int j = j0 + k;
            id[k] = 0;
            if (j < c) {
                id[k] = ids[j];
                const bool start = (j == 0) ? !(run_len > 0 && id[k] == run_a + run_len) : (id[k] != prev + 1u);
                if (start) smask |= 1u << k;
                prev = id[k];
            }
        }
        const int fs = smask ? j0 + __ffs(smask) - 1 : kNone;
        const int ls = smask ? j0 + 31 - __clz(smask) : -1;
        // first start at or after each lane (suffix minimum), the window's last start
        int m = fs, last = ls;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_down_sync(0xffffffffu, m, o);
            if (lane + o < 32) m = min(m, t);
            last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        }
        const int first = __shfl_sync(0xffffffffu, m, 0);
        int after = __shfl_down_sync(0xffffffffu, m, 1);  // first start in later lanes
        if (lane == 31) after = kNone;
        // lookups of this lane's complete runs (and, on lane 0, of the carried run)
        const bool carried = run_len > 0 && first != kNone;
        const uint32_t carried_len = carried ? run_len + (uint32_t)first : 0u;
        uint32_t my = (lane == 0 && carried) ? run_lookup_count(carried_len, scheme) : 0u;
        uint32_t len[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            len[k] = 0;
            if ((smask >> k) & 1u) {
                const uint32_t later = smask & ~((2u << k) - 1u);
                const int next = later ? j0 + __ffs(later) - 1 : after;
                if (next != kNone) {
                    len[k] = (uint32_t)(next - (j0 + k));
                    my += run_lookup_count(len[k], scheme);
                }
            }
        }
        uint32_t incl = my;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (WRITE) {
            uint64_t at = out + (incl - my);
            if (lane == 0 && carried) {
                run_lookup_write(run_a, carried_len, n, scheme, lk + at);
                at += run_lookup_count(carried_len, scheme);
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (len[k]) {
                    run_lookup_write(id[k], len[k], n, scheme, lk + at);
                    at += run_lookup_count(len[k], scheme);
                }
        }
        out += __shfl_sync(0xffffffffu, incl, 31);
        // the window's last start opens a run that may continue
        if (last >= 0) {
            run_a = ids[last];
            run_len = (uint32_t)(c - last);
        } else {
            run_len += (uint32_t)c;
        }
    }

    // Close the node's last run.
    template <bool WRITE>
    __device__ __forceinline__ void finish(int lane, uint32_t n, uint32_t *lk) {
        if (run_len > 0) {
            if (WRITE && lane == 0) run_lookup_write(run_a, run_len, n, scheme, lk + out);
            out += run_lookup_count(run_len, scheme);
            run_len = 0;
        }
    }
};

}  // namespace
}  // namespace vga
