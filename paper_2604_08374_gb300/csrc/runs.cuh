// runs.cuh -- run tracking over LEB128 lists for the run-aware union's range
// lookups (see runs.cu): the lane-serial window scan of graph validation,
// which checks the format and counts every node's lookups in one pass, and the
// byte-mask run extractor of the pass that writes them (SwarRuns).
#pragma once

#include "vga_common.cuh"

namespace vga {
namespace {

// Window width w and region slot of the lookups covering a run of length L:
// the widest kept window not longer than the run (scheme 0: 2^floor(log2 L)
// up to 16; scheme 1: 1, 4 or 16).  ceil(L / w) windows cover it, the last
// one ending at the run's end.
__device__ __forceinline__ void run_window(uint32_t L, int scheme, uint32_t &w, uint32_t &slot, uint32_t &k) {
    if (scheme == 0) {
        k = L < 16u ? 31u - __clz(L) : 4u;
        slot = k;
    } else {
        slot = L < 4u ? 0u : (L < 16u ? 1u : 2u);
        k = 2u * slot;
    }
    w = 1u << k;
}
__device__ __forceinline__ void run_window(uint32_t L, int scheme, uint32_t &w, uint32_t &slot) {
    uint32_t k;
    run_window(L, scheme, w, slot, k);
}

// Number of lookups covering the run [a, a + L): ceil(L / w), w = 2^k.
__device__ __forceinline__ uint32_t run_lookup_count(uint32_t L, int scheme) {
    uint32_t w, slot, k;
    run_window(L, scheme, w, slot, k);
    return (L + w - 1u) >> k;
}

// Lookups covering the run [a, a + L) as table row indices slot * n + i.
__device__ __forceinline__ void run_lookup_write(uint32_t a, uint32_t L, uint32_t n, int scheme, uint32_t *out) {
    uint32_t w, slot, k;
    run_window(L, scheme, w, slot, k);
    const uint32_t c = (L + w - 1u) >> k;
    const uint32_t base = slot * n + a;
    for (uint32_t j = 0; j + 1u < c; j++) out[j] = base + w * j;
    out[c - 1u] = base + L - w;
}

// Four flag bits from the top bits of a word's bytes (bit k = bit 7 of byte k).
__device__ __forceinline__ uint32_t byte_tops(uint32_t w) {
    return (((w & 0x80808080u) >> 7) * 0x00204081u) >> 21 & 0xFu;
}

// Run extraction for the lookup write pass, 128 bytes of a validated list per
// warp step, without decoding every varint.  Lane L takes the aligned word at
// window start + 4 L.  A byte ends a varint when its top bit is clear; a
// varint continues the current run exactly when it is the single byte 0x01
// following another varint's last byte (a delta of 1), except the list's first
// varint, which is an absolute id and always starts a run.  Only the varints
// that start runs are assembled (from this lane's word and the one before);
// warp scans of the deltas and of the varint counts give each start its id
// and its index, the next start in a later lane comes from a suffix minimum,
// and each lane emits the lookups of the runs that end in this window (lane 0
// also those of the run carried into it).  State carried across windows, the
// same in every lane: the id before the window, the open run, the word before
// the window and whether the list's first varint is still ahead.
struct SwarRuns {
    uint32_t id_base = 0;              // id of the last varint before the window (0 before the first)
    uint32_t run_a = 0, run_len = 0;   // the open run: first id and ids so far (run_len 0: none)
    uint32_t prev_word = 0;            // the 4 bytes before the window
    bool first_pending = true;         // the list's first varint not reached yet
    uint64_t out = 0;                  // lookups emitted so far (WRITE: next index into lk)
    int scheme = 0;

    // runs completed in one window: at most 4 per lane and the carried one
    static constexpr uint32_t kRunsCap = 132;

    // `runs`: this warp's 3 x kRunsCap words of shared memory (WRITE).
    template <bool WRITE>
    __device__ __forceinline__ void window(const uint8_t *__restrict__ bytes, uint64_t w0, uint64_t pos,
                                           uint64_t end, int lane, uint32_t n, uint32_t *lk, uint32_t *runs) {
        constexpr uint32_t kNone = 0xffffffffu;
        const uint64_t p0 = w0 + 4ull * (uint32_t)lane;
        // the byte buffer carries 256 bytes of padding past the last list
        const uint32_t w = *reinterpret_cast<const uint32_t *>(bytes + p0);
        uint32_t pw = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0) pw = prev_word;
        prev_word = __shfl_sync(0xffffffffu, w, 31);
        // bytes of this lane inside [pos, end)
        const uint32_t lo = pos > p0 ? (pos - p0 < 4u ? (uint32_t)(pos - p0) : 4u) : 0u;
        const uint32_t hi = end > p0 ? (end - p0 < 4u ? (uint32_t)(end - p0) : 4u) : 0u;
        const uint32_t in4 = hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
        const uint32_t top = byte_tops(w), ptop = byte_tops(pw);
        const uint32_t T = in4 & ~top;                                   // varint ends
        const uint32_t one = byte_tops(__vcmpeq4(w, 0x01010101u));        // bytes equal to 0x01
        const uint32_t prevT = ((~top << 1) | (~ptop >> 3 & 1u)) & 0xFu;  // the byte before ends a varint
        uint32_t firstbit = 0;
        if (first_pending) {
            const uint32_t any = __ballot_sync(0xffffffffu, T != 0u);
            if (any) {
                first_pending = false;
                if (lane == __ffs(any) - 1) firstbit = T & (0u - T);
            }
        }
        const uint32_t C = T & one & prevT & ~firstbit;  // delta 1: the run goes on
        const uint32_t S = T & ~C;                       // run starts
        // values of the starts, from the 8 bytes (pw, w); the loops below walk
        // only the set bits of S (most lanes hold none or one start)
        const uint64_t w8 = ((uint64_t)w << 32) | pw;
        const uint32_t ends8 = ((~top & 0xFu) << 4) | (~ptop & 0xFu);
        auto start_value = [&](int k) -> uint32_t {
            const int t = 4 + k;
            const uint32_t before = ends8 & ((1u << t) - 1u);
            const int sb = before ? 32 - __clz(before) : 0;  // first byte of the varint
            const int len = min(t - sb + 1, 5);               // at most 5 in a validated list
            const uint64_t x = (w8 >> (8 * sb)) & (0xFFFFFFFFFFull >> (8 * (5 - len)));
            return (uint32_t)((x & 0x7Full) | ((x >> 1) & 0x3F80ull) | ((x >> 2) & 0x1FC000ull) |
                              ((x >> 3) & 0xFE00000ull) | ((x >> 4) & 0xF0000000ull));
        };
        uint32_t dsum = __popc(C);
        for (uint32_t ms = S; ms; ms &= ms - 1u) dsum += start_value(__ffs(ms) - 1);
        // scans: deltas (ids), varint counts, and run entries (this lane's
        // starts, plus the carried run on lane 0)
        const bool has_carry = run_len > 0;  // a run is open (it may stay open)
        const uint32_t nent = __popc(S) + ((lane == 0 && has_carry) ? 1u : 0u);
        uint32_t incl_d = dsum, incl_t = __popc(T), incl_e = nent;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a = __shfl_up_sync(0xffffffffu, incl_d, o);
            const uint32_t b = __shfl_up_sync(0xffffffffu, incl_t, o);
            const uint32_t c = __shfl_up_sync(0xffffffffu, incl_e, o);
            if (lane >= o) {
                incl_d += a;
                incl_t += b;
                incl_e += c;
            }
        }
        const uint32_t vbase = incl_t - __popc(T);  // varints of the window before this lane
        const uint32_t total_t = __shfl_sync(0xffffffffu, incl_t, 31);
        // index of this lane's first start, then the first start in later lanes
        const uint32_t fsv = S ? vbase + __popc(T & ((S & (0u - S)) - 1u)) : kNone;
        uint32_t m = fsv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_down_sync(0xffffffffu, m, o);
            if (lane + o < 32) m = min(m, x);
        }
        const uint32_t first_sv = __shfl_sync(0xffffffffu, m, 0);
        uint32_t after = __shfl_down_sync(0xffffffffu, m, 1);
        if (lane == 31) after = kNone;
        // run entries in window order into `runs` (first id, length, then its
        // lookup count; the window's last start stays open: no lookups yet)
        const bool carried = has_carry && first_sv != kNone;
        const uint32_t carried_len = carried ? run_len + first_sv : 0u;
        uint32_t slot = incl_e - nent;
        uint32_t my = 0;
        uint32_t last_id = 0, last_ix = 0;  // this lane's last start
        if (lane == 0 && has_carry) {
            const uint32_t c = carried ? run_lookup_count(carried_len, scheme) : 0u;
            if (WRITE) {
                runs[slot] = run_a;
                runs[kRunsCap + slot] = carried_len;
                runs[2 * kRunsCap + slot] = c;
            }
            my += c;
            slot++;
        }
        {
            uint32_t rid = id_base + incl_d - dsum;  // id of the varint before this lane's first
            uint32_t cbits = C;
            for (uint32_t ms = S; ms; ms &= ms - 1u) {
                const int k = __ffs(ms) - 1;
                const uint32_t below = (1u << k) - 1u;
                rid += __popc(cbits & below) + start_value(k);
                cbits &= ~((2u << k) - 1u);
                const uint32_t ix = vbase + __popc(T & below);
                const uint32_t later = ms & ~((2u << k) - 1u);
                const uint32_t nx = later ? vbase + __popc(T & ((later & (0u - later)) - 1u)) : after;
                const uint32_t c = nx != kNone ? run_lookup_count(nx - ix, scheme) : 0u;
                if (WRITE) {
                    runs[slot] = rid;
                    runs[kRunsCap + slot] = nx != kNone ? nx - ix : 0u;
                    runs[2 * kRunsCap + slot] = c;
                }
                my += c;
                slot++;
                last_id = rid;
                last_ix = ix;
            }
        }
        uint32_t incl_o = my;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl_o, o);
            if (lane >= o) incl_o += x;
        }
        const uint32_t total_o = __shfl_sync(0xffffffffu, incl_o, 31);
        if (WRITE && total_o) {
            // each entry's lookup count becomes its first lookup, then every lane
            // writes lookups o = lane, lane + 32, ... of the window, finding its
            // run by binary search (the last entry whose first lookup is <= o: an
            // entry without lookups shares its offset with the next one, or is
            // the window's last, past every o): consecutive lanes store
            // consecutive lookups
            uint32_t at = incl_o - my;
            for (uint32_t e = incl_e - nent; e < incl_e; e++) {
                const uint32_t c = runs[2 * kRunsCap + e];
                runs[2 * kRunsCap + e] = at;
                at += c;
            }
            __syncwarp();
            const uint32_t total_e = __shfl_sync(0xffffffffu, incl_e, 31);
            for (uint32_t o = lane; o < total_o; o += 32) {
                uint32_t lo_r = 0, span = total_e;
                while (span > 1) {
                    const uint32_t half = span >> 1;
                    if (runs[2 * kRunsCap + lo_r + half] <= o) lo_r += half;
                    span -= half;
                }
                const uint32_t a = runs[lo_r], L = runs[kRunsCap + lo_r], j = o - runs[2 * kRunsCap + lo_r];
                uint32_t w, sl, lw;
                run_window(L, scheme, w, sl, lw);
                const uint32_t c = (L + w - 1u) >> lw;
                lk[out + o] = sl * n + (j + 1u < c ? a + w * j : a + L - w);
            }
            __syncwarp();
        }
        out += total_o;
        // the window's last start opens the run carried onward
        const uint32_t with = __ballot_sync(0xffffffffu, S != 0u);
        if (with) {
            const int hl = 31 - __clz(with);
            run_a = __shfl_sync(0xffffffffu, last_id, hl);
            run_len = total_t - __shfl_sync(0xffffffffu, last_ix, hl);
        } else if (run_len > 0) {
            run_len += total_t;
        }
        id_base += __shfl_sync(0xffffffffu, incl_d, 31);
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
    uint64_t out = 0;                 // lookups counted so far
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
// first run start after it; each lane then counts the lookups of the runs
// that start among its varints, in run order.  A varint
// is a run start unless its delta is 1 (the id right after the previous one);
// the first id of the list always starts a run.  base is the id before the
// window (updated to the last id in it); rc carries the open run.  CHECK
// tests every rule of the format (varint of at most 5 bytes and 32 bits, no
// zero delta after the list's first entry, id < n, id != self).
template <bool CHECK>
__device__ __forceinline__ Window16 scan_window16(const uint8_t *__restrict__ bytes, uint64_t pos, uint64_t end,
                                                  uint64_t &base, bool list_start, uint32_t n, uint32_t self,
                                                  int scheme, RunCarry &rc, int lane) {
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
__device__ __forceinline__ void finish_runs(RunCarry &rc, int scheme) {
    if (rc.run_len > 0) {
        rc.out += run_lookup_count(rc.run_len, scheme);
        rc.run_len = 0;
    }
}

}  // namespace
}  // namespace vga
