// runs.cuh -- LEB128 window decoding with run tracking for the run-aware
// union's range lookups (see runs.cu): shared by graph validation, which
// checks the format and counts every node's lookups in one pass, and the pass
// that writes them.
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

// Window decoder of the lookup write pass: each lane takes 4 bytes, so a warp
// decodes 128 bytes per step, and the ids come out in order for RunTracker
// (one id per lane per 32, so each run's lookups are written by one lane with
// little divergence; the lane-serial scan_window16 below is faster for
// validation but not for writing).  The window starts at a varint boundary `pos`; lane L
// holds window bytes 4L .. 4L+3 (two aligned 32-bit loads per lane shared
// through a shuffle, then a funnel shift; the byte buffer carries 256 bytes
// of padding).  Every varint that ends in the window is assembled from at
// most 5 bytes (its own lane and the one before), the deltas are prefix-
// summed across the warp, and the ids are written in order to ids[0 ..
// count).  Returns count; advance = bytes consumed up to the window's last
// complete varint (0 if none); next_base = its id.  CHECK also tests every
// rule of the format (varint of at most 5 bytes and 32 bits, no zero delta
// after a list's first entry, id < n, id != self) and sets fail on any
// break; list_start says the window begins the node's list.  (Validation
// uses scan_window16; this decoder serves the write pass on validated
// graphs.)
template <class Id, bool CHECK>
__device__ __forceinline__ int decode_window4(const uint8_t *__restrict__ bytes, uint64_t pos, uint64_t end,
                                              Id base, int lane, uint32_t *ids, int &advance, Id &next_base,
                                              bool list_start, uint64_t n, uint64_t self, bool &fail) {
    const uint64_t a0 = pos & ~3ull;
    const uint32_t *aw = reinterpret_cast<const uint32_t *>(bytes + a0);
    const uint32_t w = __ldg(aw + lane);
    uint32_t wn = __shfl_down_sync(0xffffffffu, w, 1);
    if (lane == 31) wn = __ldg(aw + 32);
    const uint32_t word = __funnelshift_r(w, wn, (uint32_t)(pos & 3ull) * 8u);
    const uint32_t prev_word = __shfl_up_sync(0xffffffffu, word, 1);
    const uint32_t pw = lane ? prev_word : 0u;  // window bytes 4L-4 .. 4L-1 (none before the window)
    // terminator bits of this lane's bytes inside [pos, end): bit 7 clear
    const uint64_t rem64 = end - pos;
    const int rem = rem64 < 128u ? (int)rem64 : 128;
    const int mine = min(max(rem - 4 * lane, 0), 4);
    const uint32_t hb = ~word & 0x80808080u;
    uint32_t tm = ((hb >> 7) | (hb >> 14) | (hb >> 21) | (hb >> 28)) & ((1u << mine) - 1u);
    // last terminator before this lane's bytes (window position), -1 if none
    int pt = tm ? 4 * lane + (31 - __clz(tm)) : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, pt, o);
        if (lane >= o) pt = max(pt, t);
    }
    const int last_all = __shfl_sync(0xffffffffu, pt, 31);
    int prev = __shfl_up_sync(0xffffffffu, pt, 1);
    if (lane == 0) prev = -1;
    // assemble this lane's varints
    uint32_t val[4];
    Id lane_sum = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        val[k] = 0;
        if ((tm >> k) & 1u) {
            const int q = 4 * lane + k;  // terminator position
            const int len = q - prev;    // bytes prev+1 .. q
            uint64_t v = 0;
            // the varint's bytes, first (least significant group) lowest, taken from
            // the previous lane's word and this one; then its 7-bit groups packed
            const int sb = prev + 1 - 4 * lane + 4;  // first byte within (pw, word): 0 .. 7
            if (len <= 4) {
                const uint32_t x = (sb < 4 ? __funnelshift_r(pw, word, 8u * (uint32_t)sb) : word >> (8 * (sb - 4))) &
                                   (0xFFFFFFFFu >> (32 - 8 * len));
                v = (x & 0x7Fu) | ((x >> 1) & 0x3F80u) | ((x >> 2) & 0x1FC000u) | ((x >> 3) & 0xFE00000u);
            } else if (len == 5) {
                const uint64_t x = ((((uint64_t)word << 32) | pw) >> (8 * sb)) & 0xFFFFFFFFFFull;
                v = (x & 0x7Full) | ((x >> 1) & (0x7Full << 7)) | ((x >> 2) & (0x7Full << 14)) |
                    ((x >> 3) & (0x7Full << 21)) | ((x >> 4) & (0x7Full << 28));
            } else {
                bad = true;
            }
            if (v > 0xFFFFFFFFull) bad = true;
            val[k] = (uint32_t)v;
            lane_sum += (Id)(uint32_t)v;
            prev = q;
        }
    }
    // prefix sums of the deltas and of the varint counts across lanes
    Id incl = lane_sum;
    int cnt_incl = __popc(tm);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Id t = __shfl_up_sync(0xffffffffu, incl, o);
        const int c = __shfl_up_sync(0xffffffffu, cnt_incl, o);
        if (lane >= o) {
            incl += t;
            cnt_incl += c;
        }
    }
    Id id = base + incl - lane_sum;
    int idx = cnt_incl - __popc(tm);
    bool f = bad;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if ((tm >> k) & 1u) {
            id += (Id)val[k];
            if (CHECK) {
                if (val[k] == 0u && !(list_start && idx == 0)) f = true;  // duplicate neighbour
                if ((uint64_t)id >= n || (uint64_t)id == self) f = true;
            }
            ids[idx++] = (uint32_t)id;
        }
    }
    if (CHECK) fail = __any_sync(0xffffffffu, f);
    advance = last_all + 1;
    next_base = base + __shfl_sync(0xffffffffu, incl, 31);
    return __shfl_sync(0xffffffffu, cnt_incl, 31);
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

// Run state of a node's list carried from one window to the next (the same in
// every lane).
struct RunCarry {
    uint32_t run_a = 0, run_len = 0;  // the run still open (run_len 0: none)
    uint64_t out = 0;                 // lookups emitted so far (WRITE: next index into lk)
};

struct Window16 {
    int count = 0;          // varints completed in the window
    uint32_t advance = 0;   // bytes consumed from pos, up to the last complete varint
    bool fail = false;      // CHECK: a rule of the format is broken
};

// One 512-byte window of a node's LEB128 list, lane-serial: lane L takes the
// 16 bytes at (pos rounded down to 16) + 16 L with one aligned 16-byte load and
// walks them in order, assembling the varints that end there (a varint that
// began in the previous lane gets that lane's trailing bytes by a shuffle).
// Warp scans give every lane the index and id of its first varint and the
// first run start after it; each lane then counts (and, WRITE, writes) the
// lookups of the runs that start among its varints, in run order.  A varint
// is a run start unless its delta is 1 (the id right after the previous one);
// the first id of the list always starts a run.  base is the id before the
// window (updated to the last id in it); rc carries the open run.  CHECK
// tests every rule of the format (varint of at most 5 bytes and 32 bits, no
// zero delta after the list's first entry, id < n, id != self).
template <bool CHECK, bool WRITE>
__device__ __forceinline__ Window16 scan_window16(const uint8_t *__restrict__ bytes, uint64_t pos, uint64_t end,
                                                  uint64_t &base, bool list_start, uint32_t n, uint32_t self,
                                                  int scheme, uint32_t *lk, RunCarry &rc, int lane) {
    constexpr int kNone = 0x7fffffff;
    Window16 W;
    const uint64_t A = pos & ~15ull;
    const int off = (int)(pos - A);
    const uint64_t g0 = A + 16ull * (uint32_t)lane;
    uint32_t w[4] = {0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u};
    if (g0 < end) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(bytes + g0));
        w[0] = x.x;
        w[1] = x.y;
        w[2] = x.z;
        w[3] = x.w;
    }
    // this lane's bytes inside [pos, end), then its terminators (bit 7 clear)
    const int lo = lane == 0 ? off : 0;
    const int hi = g0 >= end ? 0 : (int)((end - g0) < 16u ? end - g0 : 16u);
    const uint32_t vm = hi > lo ? (((1u << hi) - 1u) & ~((1u << lo) - 1u)) : 0u;
    uint32_t tm = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t hb = ~w[k] & 0x80808080u;
        tm |= (((hb >> 7) | (hb >> 14) | (hb >> 21) | (hb >> 28)) & 0xFu) << (4 * k);
    }
    tm &= vm;
    // 1. the varints ending in this lane; the first one may have begun in the previous lane
    uint32_t val_at[16];
    uint64_t acc = 0;
    int glen = 0;
    int first_i = -1;
    uint64_t first_acc = 0;
    int first_len = 0;
    bool bad = false;
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        val_at[i] = 0;
        if ((vm >> i) & 1u) {
            const uint32_t b = (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
            if (glen < 5) acc |= (uint64_t)(b & 0x7Fu) << (7 * glen);
            glen++;
            if (!(b & 0x80u)) {
                if (first_i < 0) {
                    first_i = i;
                    first_acc = acc;
                    first_len = glen;
                } else {
                    if (glen > 5 || acc > 0xFFFFFFFFull) bad = true;
                    val_at[i] = (uint32_t)acc;
                    sum += (uint32_t)acc;
                }
                acc = 0;
                glen = 0;
            }
        }
    }
    uint64_t tail_acc = __shfl_up_sync(0xffffffffu, acc, 1);
    int tail_len = __shfl_up_sync(0xffffffffu, glen, 1);
    if (lane == 0) {
        tail_acc = 0;
        tail_len = 0;
    }
    uint32_t val_first = 0;
    if (first_i >= 0) {
        const int len = tail_len + first_len;
        const uint64_t v = tail_len <= 5 ? (tail_acc | (first_acc << (7 * tail_len))) : ~0ull;
        if (len > 5 || v > 0xFFFFFFFFull) bad = true;
        val_first = (uint32_t)v;
        sum += val_first;
    }
    // 2. warp scans: index and id of the lane's first varint
    const int c = __popc(tm);
    int c_incl = c;
    uint64_t s_incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int tc = __shfl_up_sync(0xffffffffu, c_incl, o);
        const uint64_t ts = __shfl_up_sync(0xffffffffu, s_incl, o);
        if (lane >= o) {
            c_incl += tc;
            s_incl += ts;
        }
    }
    const int idx0 = c_incl - c;
    const int total = __shfl_sync(0xffffffffu, c_incl, 31);
    const uint64_t id0 = base + (s_incl - sum);
    // run starts among this lane's varints
    uint32_t smask = 0;
#pragma unroll
    for (int i = 0; i < 16; i++)
        if ((tm >> i) & 1u) {
            const uint32_t v = i == first_i ? val_first : val_at[i];
            if (v != 1u) smask |= 1u << i;
        }
    if (list_start && idx0 == 0 && first_i >= 0) smask |= 1u << first_i;
    const int fs = smask ? idx0 + __popc(tm & ((1u << (__ffs(smask) - 1)) - 1u)) : kNone;
    const int ls = smask ? idx0 + __popc(tm & ((1u << (31 - __clz(smask))) - 1u)) : -1;
    const int lt = tm ? 16 * lane + 31 - __clz(tm) : -1;  // last terminator, window position
    int m = fs, last = ls, last_t = lt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(0xffffffffu, m, o);
        if (lane + o < 32) m = min(m, t);
        last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        last_t = max(last_t, __shfl_xor_sync(0xffffffffu, last_t, o));
    }
    const int first = __shfl_sync(0xffffffffu, m, 0);
    int after = __shfl_down_sync(0xffffffffu, m, 1);  // first start in later lanes
    if (lane == 31) after = kNone;
    // 3. checks, and the lookups of the runs starting here (the carried run on lane 0)
    const bool carried = rc.run_len > 0 && first != kNone;
    uint32_t my = (lane == 0 && carried) ? run_lookup_count(rc.run_len + (uint32_t)first, scheme) : 0u;
    uint64_t id = id0;
    int idx = idx0, ps_idx = -1;
    uint32_t ps_id = 0;
    bool f = bad;
#pragma unroll
    for (int i = 0; i < 16; i++)
        if ((tm >> i) & 1u) {
            const uint32_t v = i == first_i ? val_first : val_at[i];
            id += v;
            if (CHECK) {
                if (v == 0u && !(list_start && idx == 0)) f = true;  // duplicate neighbour
                if (id >= (uint64_t)n || id == (uint64_t)self) f = true;
            }
            if ((smask >> i) & 1u) {
                if (ps_idx >= 0) my += run_lookup_count((uint32_t)(idx - ps_idx), scheme);
                ps_idx = idx;
                ps_id = (uint32_t)id;
            }
            idx++;
        }
    if (ps_idx >= 0 && after != kNone) my += run_lookup_count((uint32_t)(after - ps_idx), scheme);
    uint32_t my_incl = my;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, my_incl, o);
        if (lane >= o) my_incl += t;
    }
    if (WRITE) {
        uint64_t at = rc.out + (my_incl - my);
        if (lane == 0 && carried) {
            run_lookup_write(rc.run_a, rc.run_len + (uint32_t)first, n, scheme, lk + at);
            at += run_lookup_count(rc.run_len + (uint32_t)first, scheme);
        }
        uint64_t idw = id0;
        int ix = idx0, px = -1;
        uint32_t pid = 0;
#pragma unroll
        for (int i = 0; i < 16; i++)
            if ((tm >> i) & 1u) {
                idw += i == first_i ? val_first : val_at[i];
                if ((smask >> i) & 1u) {
                    if (px >= 0) {
                        run_lookup_write(pid, (uint32_t)(ix - px), n, scheme, lk + at);
                        at += run_lookup_count((uint32_t)(ix - px), scheme);
                    }
                    px = ix;
                    pid = (uint32_t)idw;
                }
                ix++;
            }
        if (px >= 0 && after != kNone) run_lookup_write(pid, (uint32_t)(after - px), n, scheme, lk + at);
    }
    rc.out += __shfl_sync(0xffffffffu, my_incl, 31);
    // 4. the window's last start opens a run that may continue
    if (last >= 0) {
        const int owner = __ffs(__ballot_sync(0xffffffffu, ls == last)) - 1;
        rc.run_a = __shfl_sync(0xffffffffu, ps_id, owner);
        rc.run_len = (uint32_t)(total - last);
    } else {
        rc.run_len += (uint32_t)total;
    }
    base += __shfl_sync(0xffffffffu, s_incl, 31);
    W.count = total;
    W.advance = last_t >= 0 ? (uint32_t)(last_t + 1 - off) : 0u;
    if (CHECK) W.fail = __any_sync(0xffffffffu, f);
    return W;
}

// Close a node's last run (after its last window).
template <bool WRITE>
__device__ __forceinline__ void finish_runs(RunCarry &rc, int lane, uint32_t n, int scheme, uint32_t *lk) {
    if (rc.run_len > 0) {
        if (WRITE && lane == 0) run_lookup_write(rc.run_a, rc.run_len, n, scheme, lk + rc.out);
        rc.out += run_lookup_count(rc.run_len, scheme);
        rc.run_len = 0;
    }
}

}  // namespace
}  // namespace vga
