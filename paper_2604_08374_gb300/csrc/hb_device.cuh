// hb_device.cuh -- device code shared by the single-graph kernels
// (hyperball.cu) and the batched engine (engine.cu): hashing, the slice gather
// and bytewise max, the per-node union (per neighbour and per run), the HLL
// estimator with Eq. sumD, and the mean-depth epilogue.  Everything is in an
// anonymous namespace, so each translation unit gets its own copy.
#pragma once

#include "vga_common.cuh"

namespace vga {
namespace {

// SplitMix64 (Steele, Lea, Flood 2014): one golden-ratio state step, then the
// output mix.  Sec. 3.3 inserts node v into its own counter with this hash.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}


// Lane mapping of a slice gather: each lane moves CH bytes of a neighbour's
// S-byte slice (32 bytes, one 256-bit load, from S = 32 on), G lanes cover one
// neighbour, P neighbours share one warp-wide load instruction, U loads per
// lane are in flight.
template <int S>
struct GatherShape {
    static constexpr int CH = (S >= 1024) ? S / 32 : (S >= 32 ? 32 : 16);
    static constexpr int G = S / CH;
    static constexpr int P = 32 / G;
    static constexpr int V4 = CH / 16;
    static constexpr int U = (V4 == 1) ? 4 : 2;
};

// One lane's CH bytes of a register row (16-byte aligned; 32-byte aligned when
// V4 == 2, where a single 256-bit read-only load moves them).  The rows are
// not written while the loading kernel reads them (or, in the batched engine,
// are published before the lookups that address them are read).
template <int V4>
__device__ __forceinline__ void load_row_chunk(const uint8_t *p, uint4 (&x)[V4]) {
    if constexpr (V4 == 2) {
        asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(x[0].x), "=r"(x[0].y), "=r"(x[0].z), "=r"(x[0].w), "=r"(x[1].x), "=r"(x[1].y), "=r"(x[1].z),
              "=r"(x[1].w)
            : "l"(p));
    } else {
#pragma unroll
        for (int q = 0; q < V4; q++) x[q] = __ldg(reinterpret_cast<const uint4 *>(p) + q);
    }
}

// Register maximum through 16-bit lanes.  For a register word w = [b3 b2 b1 b0]
// of uint8 registers, an unsigned max over u16x2 lanes of w keeps max(b3) and
// max(b1) in the lanes' high bytes (the high byte decides the comparison; the
// low byte is whatever came with the winner), and the same over w << 8 keeps
// max(b2) and max(b0).  Two DPX three-way maxima (__vimax3_u16x2) thus fold two
// gathered words into the running maximum, instead of the multi-instruction
// __vmaxu4 emulation.  With 4-bit registers (two per byte, the paper's packed
// format) the same holds for the top nibble of each 16-bit lane, so four
// shifted copies (w, w << 4, w << 8, w << 12) cover the four nibble positions.
// RegFmt<NIB>::Acc holds the shifted maxima of one register word.
template <bool NIB>
struct RegFmt {
    static constexpr int K = NIB ? 4 : 2;  // shifted copies per word
    static constexpr int SHIFT = NIB ? 4 : 8;
    struct Acc {
        uint32_t h[K];
    };
    static __device__ __forceinline__ void fold2(Acc &a, uint32_t w0, uint32_t w1) {
#pragma unroll
        for (int k = 0; k < K; k++) a.h[k] = __vimax3_u16x2(a.h[k], w0 << (SHIFT * k), w1 << (SHIFT * k));
    }
    // register values of the word: copy k holds, in each lane's top field, the
    // field that sat k positions lower
    static __device__ __forceinline__ uint32_t word(const Acc &a) {
        uint32_t r = 0;
        const uint32_t top = NIB ? 0xF000F000u : 0xFF00FF00u;
#pragma unroll
        for (int k = 0; k < K; k++) r |= (a.h[k] & top) >> (SHIFT * k);
        return r;
    }
    // field-wise max of two register words
    static __device__ __forceinline__ uint32_t max_word(uint32_t a, uint32_t b) {
        if (!NIB) return __vmaxu4(a, b);
        const uint32_t lo = __vmaxu4(a & 0x0F0F0F0Fu, b & 0x0F0F0F0Fu);
        const uint32_t hi = __vmaxu4((a >> 4) & 0x0F0F0F0Fu, (b >> 4) & 0x0F0F0F0Fu);
        return lo | (hi << 4);
    }
    static __device__ __forceinline__ uint4 max4(uint4 a, uint4 b) {
        return make_uint4(max_word(a.x, b.x), max_word(a.y, b.y), max_word(a.z, b.z), max_word(a.w, b.w));
    }
};

// Fold the S-byte rows row(ids[0..cnt)) into acc (4 * V4 words per lane, split
// form).  Loads for U rows per lane are issued before any is folded.
template <int S, bool NIB, class Row>
__device__ __forceinline__ void gather_fold(const Row &row, const uint32_t *ids, int cnt, int g, int sub,
                                            typename RegFmt<NIB>::Acc (&acc)[4 * GatherShape<S>::V4]) {
    using Sh = GatherShape<S>;
    using F = RegFmt<NIB>;
    static_assert(Sh::U % 2 == 0, "loads are folded in pairs");
    for (int k0 = 0; k0 < cnt; k0 += Sh::P * Sh::U) {
        uint4 x[Sh::U][Sh::V4];
#pragma unroll
        for (int u = 0; u < Sh::U; u++) {
            const int k = k0 + u * Sh::P + g;
            if (k < cnt) {
                load_row_chunk<Sh::V4>(row(ids[k]) + sub * Sh::CH, x[u]);
            } else {
#pragma unroll
                for (int q = 0; q < Sh::V4; q++) x[u][q] = make_uint4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < Sh::U; u += 2)
#pragma unroll
            for (int q = 0; q < Sh::V4; q++) {
                F::fold2(acc[4 * q + 0], x[u][q].x, x[u + 1][q].x);
                F::fold2(acc[4 * q + 1], x[u][q].y, x[u + 1][q].y);
                F::fold2(acc[4 * q + 2], x[u][q].z, x[u + 1][q].z);
                F::fold2(acc[4 * q + 3], x[u][q].w, x[u + 1][q].w);
            }
    }
}

// Row of node id in one register slice.
template <int S>
struct SliceRow {
    const uint8_t *__restrict__ cur;
    __device__ __forceinline__ const uint8_t *operator()(uint32_t id) const { return cur + (uint64_t)id * S; }
};

// Convert the split accumulators to register bytes and fold the P lane groups
// of a warp together (every lane ends with the group maximum).
template <int S, bool NIB>
__device__ __forceinline__ void finish_groups(const typename RegFmt<NIB>::Acc (&acc)[4 * GatherShape<S>::V4],
                                              uint4 (&out)[GatherShape<S>::V4]) {
    using Sh = GatherShape<S>;
    using F = RegFmt<NIB>;
#pragma unroll
    for (int q = 0; q < Sh::V4; q++)
        out[q] = make_uint4(F::word(acc[4 * q + 0]), F::word(acc[4 * q + 1]), F::word(acc[4 * q + 2]),
                            F::word(acc[4 * q + 3]));
#pragma unroll
    for (int o = Sh::G; o < 32; o <<= 1)
#pragma unroll
        for (int q = 0; q < Sh::V4; q++) {
            uint4 y;
            y.x = __shfl_xor_sync(0xffffffffu, out[q].x, o);
            y.y = __shfl_xor_sync(0xffffffffu, out[q].y, o);
            y.z = __shfl_xor_sync(0xffffffffu, out[q].z, o);
            y.w = __shfl_xor_sync(0xffffffffu, out[q].w, o);
            out[q] = F::max4(out[q], y);
        }
}

// Alg. 1 initialisation of node v, as a key j << 8 | rho: its counter gets rho
// in register j, where j is the top p bits of the hash and rho the position of
// the first set bit of the remaining 64-p bits (65-p if none).  With 4-bit
// registers (nib) rho is clamped to 15.
__device__ __forceinline__ uint32_t node_key(uint32_t v, int p, uint64_t seed, bool nib) {
    const uint64_t h = splitmix64((uint64_t)v ^ seed);
    const uint32_t j = (uint32_t)(h >> (64 - p));
    const uint64_t w = h << p;
    uint32_t rho = w ? (uint32_t)__clzll((long long)w) + 1u : (uint32_t)(65 - p);
    if (nib && rho > 15u) rho = 15u;
    return j << 8 | rho;
}

// Store node v's initial counter into registers that were zeroed before.  With
// 4-bit registers register j is nibble j % 2 of byte j / 2 (the low nibble
// first).  A shard stores only slices [s0, s1), its slice s0 first.
__device__ __forceinline__ void init_node(uint8_t *__restrict__ regs, uint32_t n, int p, int S, uint64_t seed,
                                          uint32_t v, bool nib = false, uint32_t s0 = 0u,
                                          uint32_t s1 = 0xffffffffu) {
    const uint32_t key = node_key(v, p, seed, nib);
    const uint32_t j = key >> 8, rho = key & 0xffu;
    const uint32_t byte = nib ? j >> 1 : j;
    const uint32_t val = nib ? rho << (4u * (j & 1u)) : rho;
    const uint32_t s = byte / (uint32_t)S, o = byte % (uint32_t)S;
    if (s < s0 || s >= s1) return;  // a register-range shard holds slices [s0, s1) only
    regs[((uint64_t)(s - s0) * n + v) * (uint64_t)S + o] = (uint8_t)val;
}

// Fold the node's own slice into the gathered maximum, store it, and set
// *flag if any register changed (one atomic per warp at most); with chg given
// (the slice's change bytes), chg[v] = 1 as well.
template <int S, bool NIB>
__device__ __forceinline__ void union_store(const typename RegFmt<NIB>::Acc (&acc)[4 * GatherShape<S>::V4],
                                            const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt, uint32_t v,
                                            int lane, uint32_t *flag, uint8_t *chg = nullptr) {
    using Sh = GatherShape<S>;
    const int g = lane / Sh::G, sub = lane % Sh::G;
    uint4 nb[Sh::V4];
    finish_groups<S, NIB>(acc, nb);
    bool changed = false;
    if (g == 0) {
        const uint4 *own = reinterpret_cast<const uint4 *>(cur + (uint64_t)v * S + sub * Sh::CH);
        uint4 *dst = reinterpret_cast<uint4 *>(nxt + (uint64_t)v * S + sub * Sh::CH);
#pragma unroll
        for (int q = 0; q < Sh::V4; q++) {
            const uint4 o4 = __ldg(own + q);
            const uint4 res = RegFmt<NIB>::max4(nb[q], o4);
            dst[q] = res;
            changed |= (res.x != o4.x) | (res.y != o4.y) | (res.z != o4.z) | (res.w != o4.w);
        }
    }
    if (__any_sync(0xffffffffu, changed) && lane == 0) {
        if (*reinterpret_cast<volatile uint32_t *>(flag) == 0u) atomicOr(flag, 1u);
        if (chg) chg[v] = 1u;
    }
}

// Eq. hll-union of node v for one register slice: next[v] = max(cur[v],
// max_{w in N(v)} cur[w]) bytewise.  The warp decodes the node's LEB128 list
// 32 bytes at a time (decode_window), stages the decoded ids in `ids` (32
// entries of shared memory) and gathers each neighbour's S-byte slice.
template <int S, bool NIB = false>
__device__ __forceinline__ void union_node_edges(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes,
                                                 const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt,
                                                 uint32_t v, uint32_t *ids, int lane, uint32_t *flag,
                                                 uint8_t *chg = nullptr) {
    using Sh = GatherShape<S>;
    const int g = lane / Sh::G, sub = lane % Sh::G;
    const uint32_t lt_mask = (1u << lane) - 1u;
    typename RegFmt<NIB>::Acc acc[4 * Sh::V4] = {};
    uint64_t pos = off[v];
    const uint64_t end = off[v + 1];
    uint32_t base = 0;
    while (pos < end) {
        const WindowDecode<uint32_t> r = decode_window<uint32_t>(bytes, pos, end, base, lane);
        const uint32_t T = r.term_mask;
        if (T == 0) break;  // cannot happen on a validated graph; guarantees progress
        if ((T >> lane) & 1u) ids[__popc(T & lt_mask)] = r.id;
        __syncwarp();
        gather_fold<S, NIB>(SliceRow<S>{cur}, ids, __popc(T), g, sub, acc);
        __syncwarp();
        base = r.next_base;
        pos += (uint64_t)r.advance;
    }
    union_store<S, NIB>(acc, cur, nxt, v, lane, flag, chg);
}

// ---------------------------------------------------------------------------
// 1D TMA (cp.async.bulk) staging of a node's range lookups into shared memory.
// Each warp owns two 512-byte buffers and two mbarriers; lane 0 issues a bulk
// copy per buffer and the warp consumes one buffer while the next is in
// flight.  Source and size are 16-byte multiples: a node's range is widened to
// whole 4-lookup groups (the lookup list carries 4 entries of tail padding).
// Every wait is bounded; a wait that runs out sets *err.
// ---------------------------------------------------------------------------
constexpr int kLkChunk = 128;  // lookups per bulk copy

struct LkStage {
    uint32_t buf[2][kLkChunk];
    unsigned long long bar[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Lane 0: initialise the warp's two barriers (one arrival per phase).
__device__ __forceinline__ void lk_stage_init(LkStage &st, int lane) {
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&st.bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&st.bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}

// The lookup stream is read once per slice: its lines are marked evict-first in
// L2 so that they do not push out the slice's table region.
__device__ __forceinline__ void lk_bulk_load(LkStage &st, int slot, const uint32_t *src, uint32_t bytes) {
    const uint32_t bar = smem_u32(&st.bar[slot]);
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(st.buf[slot])),
        "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}

// Bounded wait for the phase `parity` of a barrier to complete.
__device__ __forceinline__ bool lk_wait(LkStage &st, int slot, uint32_t parity) {
    const uint32_t bar = smem_u32(&st.bar[slot]);
    uint32_t done = 0;
    for (uint32_t i = 0; i < (1u << 21) && !done; i++) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// Word-wise register max into next[v] for the chunks of a split hub:
// *p = max(*p, val) field by field, by compare-and-swap.  Every successful
// swap by another chunk only raises fields, so the loop ends after a few
// rounds; the bound (never reached) reports through *err instead of spinning.
template <bool NIB>
__device__ __forceinline__ void atomic_max_word(uint32_t *p, uint32_t val, int *err) {
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(p);
    for (int i = 0; i < 4096; i++) {
        const uint32_t want = RegFmt<NIB>::max_word(old, val);
        if (want == old) return;
        const uint32_t seen = atomicCAS(p, old, want);
        if (seen == old) return;
        old = seen;
    }
    atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// Lean row gather of the single-graph run-aware union.  Each lane moves CH
// bytes of a row (16, or 32 from S = 1024 on), G lanes cover a row, P rows
// share one warp-wide load, U rows per lane are in flight, and a lane group
// takes U consecutive entries of the staged lookup chunk, read as one vector
// from shared memory.  Compared with GatherShape this halves the accumulator
// registers (fewer bytes per lane) and keeps the same bytes in flight, so more
// warps fit an SM; full steps carry no bounds checks.
// ---------------------------------------------------------------------------
template <int S>
struct LeanShape {
    static constexpr int CH = S >= 1024 ? 32 : 16;
    static constexpr int G = S / CH;
    static constexpr int P = 32 / G;
    static constexpr int V4 = CH / 16;
    static constexpr int U = V4 == 1 ? 4 : 2;
};

// Fold the rows of entries buf[lo .. hi) of a 16-byte-aligned staged chunk
// into acc; base = the table region plus this lane's byte offset in a row.
template <int S, bool NIB>
__device__ __forceinline__ void lean_fold(const uint8_t *__restrict__ base, const uint32_t *buf, int lo, int hi, int g,
                                          typename RegFmt<NIB>::Acc (&acc)[4 * LeanShape<S>::V4]) {
    using Sh = LeanShape<S>;
    using F = RegFmt<NIB>;
    constexpr int STEP = Sh::P * Sh::U;
    auto step = [&](int kb, bool check) {
        uint32_t r[Sh::U];
        if constexpr (Sh::U == 4) {
            const uint4 t = *reinterpret_cast<const uint4 *>(buf + kb);
            r[0] = t.x;
            r[1] = t.y;
            r[2] = t.z;
            r[3] = t.w;
        } else {
            const uint2 t = *reinterpret_cast<const uint2 *>(buf + kb);
            r[0] = t.x;
            r[1] = t.y;
        }
        uint4 x[Sh::U][Sh::V4];
#pragma unroll
        for (int u = 0; u < Sh::U; u++) {
            if (!check || (kb + u >= lo && kb + u < hi)) {
                load_row_chunk<Sh::V4>(base + (uint64_t)r[u] * S, x[u]);
            } else {
#pragma unroll
                for (int q = 0; q < Sh::V4; q++) x[u][q] = make_uint4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < Sh::U; u += 2)
#pragma unroll
            for (int q = 0; q < Sh::V4; q++) {
                F::fold2(acc[4 * q + 0], x[u][q].x, x[u + 1][q].x);
                F::fold2(acc[4 * q + 1], x[u][q].y, x[u + 1][q].y);
                F::fold2(acc[4 * q + 2], x[u][q].z, x[u + 1][q].z);
                F::fold2(acc[4 * q + 3], x[u][q].w, x[u + 1][q].w);
            }
    };
    // a step covers STEP entries from a multiple of U: a head step that may
    // start below lo, full steps, a tail step that may end past hi (the
    // entries outside [lo, hi) are read from the stage but not gathered)
    int k0 = lo & ~(Sh::U - 1);
    if (k0 < lo) {
        const int kb = k0 + g * Sh::U;
        if (kb < hi) step(kb, true);
        k0 += STEP;
    }
    for (; k0 + STEP <= hi; k0 += STEP) step(k0 + g * Sh::U, false);
    if (k0 < hi) {
        const int kb = k0 + g * Sh::U;
        if (kb < hi) step(kb, true);
    }
}

// The split accumulators as register bytes, folded over the warp's P lane
// groups: every lane ends with the maximum of its CH-byte part of the row.
template <int S, bool NIB>
__device__ __forceinline__ void lean_finish(const typename RegFmt<NIB>::Acc (&acc)[4 * LeanShape<S>::V4],
                                            uint4 (&out)[LeanShape<S>::V4]) {
    using Sh = LeanShape<S>;
    using F = RegFmt<NIB>;
#pragma unroll
    for (int q = 0; q < Sh::V4; q++)
        out[q] = make_uint4(F::word(acc[4 * q + 0]), F::word(acc[4 * q + 1]), F::word(acc[4 * q + 2]),
                            F::word(acc[4 * q + 3]));
#pragma unroll
    for (int o = Sh::G; o < 32; o <<= 1)
#pragma unroll
        for (int q = 0; q < Sh::V4; q++) {
            uint4 y;
            y.x = __shfl_xor_sync(0xffffffffu, out[q].x, o);
            y.y = __shfl_xor_sync(0xffffffffu, out[q].y, o);
            y.z = __shfl_xor_sync(0xffffffffu, out[q].z, o);
            y.w = __shfl_xor_sync(0xffffffffu, out[q].w, o);
            out[q] = F::max4(out[q], y);
        }
}

// Store node v's slice row: max(its gathered maximum nb, cur[v]) into next[v]
// (by word-wise atomic max for a split hub's chunk: next[v] starts each pass at
// or below the result, so after all chunks it holds their maximum),
// setting *flag, and chg[v] when given, if a register changed.  Lanes of
// group 0 hold the row; every lane takes part in the vote.
template <int S, bool NIB>
__device__ __forceinline__ void lean_store(const uint4 (&nb)[LeanShape<S>::V4], const uint8_t *__restrict__ cur,
                                           uint8_t *__restrict__ nxt, uint32_t v, int lane, bool hub, uint32_t *flag,
                                           int *err, uint8_t *chg) {
    using Sh = LeanShape<S>;
    const int g = lane / Sh::G, sub = lane % Sh::G;
    bool changed = false;
    if (g == 0) {
        const uint4 *own = reinterpret_cast<const uint4 *>(cur + (uint64_t)v * S + sub * Sh::CH);
        uint4 *dst = reinterpret_cast<uint4 *>(nxt + (uint64_t)v * S + sub * Sh::CH);
#pragma unroll
        for (int q = 0; q < Sh::V4; q++) {
            const uint4 o4 = __ldg(own + q);
            const uint4 res = RegFmt<NIB>::max4(nb[q], o4);
            if (hub) {
                uint32_t *d = reinterpret_cast<uint32_t *>(dst + q);
                atomic_max_word<NIB>(d + 0, res.x, err);
                atomic_max_word<NIB>(d + 1, res.y, err);
                atomic_max_word<NIB>(d + 2, res.z, err);
                atomic_max_word<NIB>(d + 3, res.w, err);
            } else {
                dst[q] = res;
            }
            changed |= (res.x != o4.x) | (res.y != o4.y) | (res.z != o4.z) | (res.w != o4.w);
        }
    }
    if (__any_sync(0xffffffffu, changed) && lane == 0) {
        if (*reinterpret_cast<volatile uint32_t *>(flag) == 0u) atomicOr(flag, 1u);
        if (chg) chg[v] = 1u;
    }
}

// Streaming of an item's entries src[b .. e) through the warp's TMA stage, in
// chunks of kLkChunk entries counted from a0 = b rounded down to a multiple
// of 4 (the entries before b in that 16-byte group must be readable): the
// kernel calls stage_start once, then for chunk c = 0, 1, ...: stage_acquire,
// its own processing of buf(c), stage_release.  Chunk c holds entries
// [a0 + c kLkChunk, ...) of src.  Bounded waits; a wait that runs out sets
// *err.  (Explicit loops in the kernels, not a callback: the compiler keeps
// the fold's state in registers that way.)
struct StageStream {
    const uint32_t *src;
    uint64_t a0;
    uint32_t total;   // entries from a0, rounded up to a multiple of 4
    uint32_t chunks;
    __device__ __forceinline__ StageStream(const uint32_t *src_, uint64_t b, uint64_t e)
        : src(src_), a0(b & ~3ull), total(0), chunks(0) {
        if (e > b) {
            total = (uint32_t)(((e + 3) & ~3ull) - a0);
            chunks = (total + kLkChunk - 1) / kLkChunk;
        }
    }
    __device__ __forceinline__ void load(LkStage &st, uint32_t c) const {
        const uint32_t s0 = c * kLkChunk;
        lk_bulk_load(st, (int)(c & 1u), src + a0 + s0, min(total - s0, (uint32_t)kLkChunk) * 4u);
    }
    __device__ __forceinline__ void start(LkStage &st, int lane) const {
        if (lane == 0)
            for (uint32_t c = 0; c < 2 && c < chunks; c++) load(st, c);
    }
    // wait for chunk c (every lane observes the barrier phase itself: acquire for its reads)
    __device__ __forceinline__ const uint32_t *acquire(LkStage &st, uint32_t c, uint32_t &phase, int *err,
                                                       int lane) const {
        const int slot = (int)(c & 1u);
        if (!__all_sync(0xffffffffu, lk_wait(st, slot, (phase >> slot) & 1u))) {
            if (lane == 0) atomicExch(err, 1);
            lk_wait(st, slot, (phase >> slot) & 1u);  // give an in-flight copy a last chance
        }
        phase ^= 1u << slot;
        return st.buf[slot];
    }
    // chunk c consumed: its buffer takes chunk c + 2
    __device__ __forceinline__ void release(LkStage &st, uint32_t c, int lane) const {
        __syncwarp();
        if (lane == 0 && c + 2 < chunks) load(st, c + 2);
    }
};

// Run-aware Eq. hll-union of one work item (a whole node, or one chunk of a
// split hub) for one register slice whose table region `tab` has been built:
// the item's range lookups stream through the warp's TMA stage `st` (barrier
// phases in `phase`) and each lookup's table row is gathered (lean_fold);
// then next[v] = max(gathered, cur[v]) (lean_store).
template <int S, bool NIB>
__device__ __forceinline__ void union_item(const RunItem &it, const uint32_t *__restrict__ lk,
                                           const uint8_t *__restrict__ cur, const uint8_t *__restrict__ tab,
                                           uint8_t *__restrict__ nxt, LkStage &st, uint32_t &phase, int lane,
                                           uint32_t *flag, int *err, uint8_t *chg) {
    using Sh = LeanShape<S>;
    const uint32_t v = it.v & ~kHubChunk;
    const bool hub = (it.v & kHubChunk) != 0;
    typename RegFmt<NIB>::Acc acc[4 * Sh::V4] = {};
    const int g = lane / Sh::G;
    const uint8_t *base = tab + (lane % Sh::G) * Sh::CH;
    const StageStream ss(lk, it.b, it.b + it.cnt);
    const uint32_t off_b = (uint32_t)(it.b - ss.a0), off_e = off_b + it.cnt;
    ss.start(st, lane);
    for (uint32_t c = 0; c < ss.chunks; c++) {
        const uint32_t *buf = ss.acquire(st, c, phase, err, lane);
        const uint32_t s0 = c * kLkChunk;
        const uint32_t lo = max(off_b, s0), hi = min(off_e, s0 + (uint32_t)kLkChunk);
        if (hi > lo) lean_fold<S, NIB>(base, buf, (int)(lo - s0), (int)(hi - s0), g, acc);
        ss.release(st, c, lane);
    }
    uint4 nb[Sh::V4];
    lean_finish<S, NIB>(acc, nb);
    lean_store<S, NIB>(nb, cur, nxt, v, lane, hub, flag, err, chg);
}

// Grouped run-aware Eq. hll-union of one group of NODES consecutive nodes
// (GroupItem, runs.cu) for one register slice: the group's distinct rows
// stream through the warp's TMA stage class by class; each class's rows are
// gathered and folded into one accumulator, which at the class's end is
// reduced over the warp and max-merged into the partial rows `part` (NODES x S
// bytes of this warp's shared memory) of the class's nodes.  Finally every
// node's partial is maxed with its own registers and stored (lean_store).  The
// maximum over each node's rows is that over its own lookup list, so the
// registers equal those of union_item bit for bit.
template <int S, bool NIB, int NODES>
__device__ __forceinline__ void union_group(const GroupItem &gi, const uint32_t *__restrict__ rows,
                                            const uint2 *__restrict__ cls, const uint8_t *__restrict__ cur,
                                            const uint8_t *__restrict__ tab, uint8_t *__restrict__ nxt, uint4 *part,
                                            LkStage &st, uint32_t &phase, int lane, uint32_t *flag, int *err,
                                            uint8_t *chg) {
    using Sh = LeanShape<S>;
    using F = RegFmt<NIB>;
    constexpr int W16 = S / 16;  // uint4 words of a slice row
    const uint32_t cnt = gi.cnt, nc = gi.nc;
    const uint64_t cls0 = gi.cls;
    for (int q = lane; q < NODES * W16; q += 32) part[q] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    typename F::Acc acc[4 * Sh::V4] = {};
    const int g = lane / Sh::G, sub = lane % Sh::G;
    const uint8_t *base = tab + sub * Sh::CH;
    if (cnt > 0) {
        uint32_t ci = 0;
        uint2 cd = cls[cls0];  // {node mask, rows} of the current class
        uint32_t cend = cd.y;  // group entry where the current class ends
        const StageStream ss(rows, gi.b, gi.b + cnt);  // gi.b is a multiple of 4
        ss.start(st, lane);
        for (uint32_t c = 0; c < ss.chunks; c++) {
            const uint32_t *buf = ss.acquire(st, c, phase, err, lane);
            const uint32_t s0 = c * kLkChunk;
            uint32_t lo = s0;
            const uint32_t hi = min(cnt, s0 + (uint32_t)kLkChunk);
            while (lo < hi) {  // warp-uniform: split the chunk at class ends
                const uint32_t seg = min(hi, cend);
                if (seg > lo) lean_fold<S, NIB>(base, buf, (int)(lo - s0), (int)(seg - s0), g, acc);
                lo = seg;
                if (lo == cend) {  // the class is complete
                    uint4 w[Sh::V4];
                    lean_finish<S, NIB>(acc, w);
                    if (g == 0) {
#pragma unroll
                        for (int j = 0; j < NODES; j++)
                            if ((cd.x >> j) & 1u)
#pragma unroll
                                for (int q = 0; q < Sh::V4; q++) {
                                    uint4 &pp = part[j * W16 + sub * Sh::V4 + q];
                                    pp = F::max4(pp, w[q]);
                                }
                    }
#pragma unroll
                    for (int q = 0; q < 4 * Sh::V4; q++) acc[q] = typename F::Acc{};
                    if (++ci < nc) {
                        cd = cls[cls0 + ci];
                        cend += cd.y;
                    } else {
                        cend = 0xffffffffu;  // past the last entry: no further class end
                    }
                }
            }
            ss.release(st, c, lane);
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NODES; j++) {
        const uint32_t v = gi.node[j];  // read again here, not held in registers through the loop
        if (v == 0xffffffffu) break;
        uint4 nb[Sh::V4];
#pragma unroll
        for (int q = 0; q < Sh::V4; q++) nb[q] = part[j * W16 + sub * Sh::V4 + q];
        lean_store<S, NIB>(nb, cur, nxt, v, lane, false, flag, err, chg);
    }
}

// Keys of the first pass's scatter: node_key repacked as j << KeyFmt<K>::RHO_BITS
// | rho.  16-bit keys (p <= 10: j < 2^10, rho <= 61 < 2^6) halve the bytes the
// scatter reads; wider precisions keep the 32-bit form.
template <class K>
struct KeyFmt {
    static constexpr int RHO_BITS = sizeof(K) == 2 ? 6 : 8;
    static __device__ __forceinline__ K pack(uint32_t key32) {
        return (K)(((key32 >> 8) << RHO_BITS) | (key32 & 0xffu));
    }
    static __device__ __forceinline__ uint32_t j(uint32_t k) { return k >> RHO_BITS; }
    static __device__ __forceinline__ uint32_t rho(uint32_t k) { return k & ((1u << RHO_BITS) - 1u); }
};
constexpr int kKey16MaxP = 10;

// Pack the scatter's register cells into register words and store them for
// slices [s0, s1) of node v (by word-wise atomic max for a split hub's chunk:
// next[v] holds no register above the result when the pass starts); *flag is
// set when a stored register exceeds the node's own counter (key `own`), and
// with chg given chg[s][v] = 1 for each slice where one does.
template <bool NIB, class K>
__device__ __forceinline__ void fp_store(uint32_t own, const uint32_t *cells, uint32_t m, uint32_t v, uint32_t n,
                                         int s_log2, uint32_t s0, uint32_t s1, bool hub, uint8_t *__restrict__ nxt,
                                         int lane, uint32_t *flag, int *err, uint8_t *chg) {
    using KF = KeyFmt<K>;
    // pack: 32-bit word k holds registers 4k .. 4k+3 (bytes), or 8k .. 8k+7
    // (nibbles, the low nibble first)
    const uint32_t per_word = NIB ? 8u : 4u, words = m / per_word;
    const uint32_t own_j = KF::j(own), own_rho = KF::rho(own);
    const uint32_t S = 1u << s_log2;
    bool changed = false;
    for (uint32_t k = lane; k < words; k += 32) {
        uint32_t w;
        if (NIB) {
            const uint4 a = reinterpret_cast<const uint4 *>(cells)[2 * k];
            const uint4 b = reinterpret_cast<const uint4 *>(cells)[2 * k + 1];
            w = a.x | a.y << 4 | a.z << 8 | a.w << 12 | b.x << 16 | b.y << 20 | b.z << 24 | b.w << 28;
        } else {
            const uint4 a = reinterpret_cast<const uint4 *>(cells)[k];
            w = a.x | a.y << 8 | a.z << 16 | a.w << 24;
        }
        const uint32_t byte = 4u * k, sl = byte >> s_log2;
        if (sl < s0 || sl >= s1) continue;
        const uint32_t mine = own_j / per_word == k ? own_rho << ((32u / per_word) * (own_j % per_word)) : 0u;
        changed |= w != mine;
        if (chg && w != mine) chg[(uint64_t)(sl - s0) * n + v] = 1u;  // lanes of one slice store the same byte
        uint32_t *dst =
            reinterpret_cast<uint32_t *>(nxt + (((uint64_t)(sl - s0) * n + v) << s_log2) + (byte & (S - 1u)));
        if (hub)
            atomic_max_word<NIB>(dst, w, err);
        else
            *dst = w;
    }
    if (__any_sync(0xffffffffu, changed) && lane == 0) {
        if (*reinterpret_cast<volatile uint32_t *>(flag) == 0u) atomicOr(flag, 1u);
    }
}

// Zero the warp's m register cells and put the node's own key in; returns it.
template <class K>
__device__ __forceinline__ uint32_t fp_init(uint32_t *cells, uint32_t m, const K *__restrict__ keys, uint32_t v,
                                            int lane) {
    using KF = KeyFmt<K>;
    for (uint32_t k = lane; k < m / 4u; k += 32) reinterpret_cast<uint4 *>(cells)[k] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    const uint32_t own = __ldg(keys + v);
    if (lane == 0) cells[KF::j(own)] = KF::rho(own);
    __syncwarp();
    return own;
}

// First pass of Eq. hll-union (t = 1) as a scatter.  After the initialisation
// (Alg. 1) every counter holds one register, the node's key (node_key), so
// register j of next[v] is the largest rho among the keys of v and its
// neighbours whose register index is j: no register row needs to be gathered.
// A warp walks its work item's range lookups; a lookup r = slot * n + i of
// window width w (runs.cuh: the windows of a run stay inside it) covers the
// neighbour ids i .. i + w - 1.  The lookups of windows up to 4 ids wide and
// those of wider ones are compacted in turn through `stage` (32 words, the
// window start with its level in the top bits), so that 8 narrow or 2 wide
// lookups share a round of the warp, consecutive lanes taking consecutive
// ids; their keys are read from `keys` and folded into the warp's m
// shared-memory cells (one u32 per register) by atomicMax.  The cells are then
// packed into register words and stored for slices [s0, s1) of the slice-major
// layout (all slices, or a register-range shard's own, its slice s0 first), or
// merged word by word by atomic max for the chunk of a split hub
// (atomic_max_word; next[v] holds no register above the result when the pass
// starts).  *flag is set when a stored register exceeds the node's own
// counter, and with chg given (change bytes, [slice][N] from slice s0 on)
// chg[s][v] = 1 for each slice where one does.
template <bool NIB, class K>
__device__ __forceinline__ void first_pass_item(const RunItem it, const uint32_t *__restrict__ lk,
                                                const K *__restrict__ keys, uint32_t n, int p, int scheme,
                                                int s_log2, uint32_t s0, uint32_t s1, uint8_t *__restrict__ nxt,
                                                uint32_t *cells, uint32_t *stage, int lane, uint32_t *flag,
                                                int *err, uint8_t *chg = nullptr) {
    using KF = KeyFmt<K>;
    const uint32_t m = 1u << p;
    const uint32_t v = it.v & ~kHubChunk;
    const uint32_t own = fp_init<K>(cells, m, keys, v, lane);
    const int rows = table_rows(scheme);
    const uint64_t e = it.b + it.cnt;
    uint32_t r_next = (it.b + (uint64_t)lane < e) ? __ldcs(lk + it.b + lane) : 0u;
    for (uint64_t base = it.b; base < e; base += 32) {
        const bool valid = base + (uint64_t)lane < e;
        const uint32_t r = r_next;
        if (base + 32 + (uint64_t)lane < e) r_next = __ldcs(lk + base + 32 + lane);
        uint32_t slot = 0;
        for (int s = 1; s < rows; s++) slot += r >= (uint32_t)s * n ? 1u : 0u;
        const uint32_t level = scheme == 0 ? slot : 2u * slot;
        const uint32_t packed = (r - slot * n) | (level << 29);  // i < 2^29 (kRunMaxNodes)
#pragma unroll
        for (int grp = 0; grp < 2; grp++) {
            const int G = grp == 0 ? 4 : 16;  // lanes per lookup: windows of 1..4, of 8..16 ids
            const int per = 32 / G;
            const uint32_t mask = __ballot_sync(0xffffffffu, valid && ((level <= 2u) == (grp == 0)));
            if (!mask) continue;
            if ((mask >> lane) & 1u) stage[__popc(mask & ((1u << lane) - 1u))] = packed;
            __syncwarp();
            const int c = __popc(mask);
            const int my = lane / G;
            const uint32_t off = (uint32_t)(lane % G);
            for (int q = 0; q < c; q += 4 * per) {
                uint32_t key[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int x = q + u * per + my;
                    key[u] = 0u;  // a key is never 0 (rho >= 1)
                    if (x < c) {
                        const uint32_t sx = stage[x];
                        if (off < (1u << (sx >> 29))) key[u] = __ldg(keys + (sx & 0x1fffffffu) + off);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (key[u]) atomicMax(cells + KF::j(key[u]), KF::rho(key[u]));
            }
            __syncwarp();
        }
    }
    fp_store<NIB, K>(own, cells, m, v, n, s_log2, s0, s1, (it.v & kHubChunk) != 0, nxt, lane, flag, err, chg);
}

// First pass as a scatter for the per-neighbour variant, which has no range
// lookups: the warp decodes node v's list 32 bytes at a time (decode_window;
// ids of a run come out on consecutive lanes) and folds the keys of the
// decoded ids into its register cells, then stores like first_pass_item.
template <bool NIB, class K>
__device__ __forceinline__ void first_pass_csr(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes,
                                               const K *__restrict__ keys, uint32_t v, uint32_t n, int p, int s_log2,
                                               uint32_t s0, uint32_t s1, uint8_t *__restrict__ nxt, uint32_t *cells,
                                               int lane, uint32_t *flag, int *err, uint8_t *chg = nullptr) {
    using KF = KeyFmt<K>;
    const uint32_t m = 1u << p;
    const uint32_t own = fp_init<K>(cells, m, keys, v, lane);
    uint64_t pos = off[v];
    const uint64_t end = off[v + 1];
    uint32_t base = 0;
    while (pos < end) {
        const WindowDecode<uint32_t> r = decode_window<uint32_t>(bytes, pos, end, base, lane);
        if (r.term_mask == 0) break;  // cannot happen on a validated graph; guarantees progress
        if ((r.term_mask >> lane) & 1u) {
            const uint32_t key = __ldg(keys + r.id);
            atomicMax(cells + KF::j(key), KF::rho(key));
        }
        base = r.next_base;
        pos += (uint64_t)r.advance;
    }
    __syncwarp();
    fp_store<NIB, K>(own, cells, m, v, n, s_log2, s0, s1, false, nxt, lane, flag, err, chg);
}

// A work item whose node has no neighbour that changed in this slice during
// the previous pass keeps its registers: next[v] = cur[v] (when no neighbour u
// of v changed, max over u of cur[u] is the previous pass's max over u, which
// cur[v] already holds).  The chunk of a split hub merges cur[v] into next[v]
// by word-wise atomic max instead, since other chunks of v may be merging
// their own results at the same time.
template <int S, bool NIB>
__device__ __forceinline__ void keep_item(const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt, uint32_t v,
                                          bool hub, int lane, int *err) {
    const uint64_t row = (uint64_t)v * S;
    if (!hub) {
        for (int q = lane; q < S / 16; q += 32)
            reinterpret_cast<uint4 *>(nxt + row)[q] = __ldg(reinterpret_cast<const uint4 *>(cur + row) + q);
    } else {
        for (int q = lane; q < S / 4; q += 32)
            atomic_max_word<NIB>(reinterpret_cast<uint32_t *>(nxt + row) + q,
                                 __ldg(reinterpret_cast<const uint32_t *>(cur + row) + q), err);
    }
}

// Rows of one slice's sparse table built by one CTA (`table_item`), and the
// shared memory that takes them with their 15-row halo.
template <int S>
struct TableShape {
    static constexpr int B = (S >= 1024) ? 16 : 32;
    static constexpr int R = B + 15;
    static constexpr int C16 = S / 16;  // 16-byte chunks per row
};
constexpr int kTableSmemBytes = (16 + 15) * 1024;  // largest (B + 15) * S

// Table-region rows [r0, r0 + B) of one slice, straight from the slice's
// counters: T_0[i] = cur[i] and T_k[i] = max(cur[i .. i + 2^k)) for the
// scheme's levels k (scheme 0: 1..4; scheme 1: 2 and 4) and the rows with
// i + 2^k <= n.  The rows and their halo are staged once in `buf`; each thread
// then owns one 16-byte chunk of one output row, copies it to T_0 and folds
// the 16 rows of its widest window, writing each kept level as the window
// reaches 2^k rows (at tab + slot * n * S; scheme 0: slot k, scheme 1: slot
// k / 2).  All threads of the CTA (256) take part.
template <int S, bool NIB = false>
__device__ void table_item(const uint8_t *__restrict__ cur, uint8_t *__restrict__ tab, uint32_t n, uint32_t r0,
                           uint8_t *buf, int scheme = 0) {
    using T = TableShape<S>;
    uint4 *b4 = reinterpret_cast<uint4 *>(buf);
    const uint32_t avail = (n - r0 < (uint32_t)T::R) ? n - r0 : (uint32_t)T::R;
    for (int x = threadIdx.x; x < T::R * T::C16; x += blockDim.x) {
        const uint32_t row = x / T::C16, c = x % T::C16;
        b4[x] = (row < avail) ? __ldg(reinterpret_cast<const uint4 *>(cur + (uint64_t)(r0 + row) * S) + c)
                              : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < T::B * T::C16; x += blockDim.x) {
        const uint32_t row = x / T::C16, c = x % T::C16;
        const uint64_t i = (uint64_t)r0 + row;
        uint4 acc = b4[x];
        if (i < n) reinterpret_cast<uint4 *>(tab + i * S)[c] = acc;
#pragma unroll
        for (int j = 1; j < 16; j++) {
            acc = RegFmt<NIB>::max4(acc, b4[x + j * T::C16]);
            if ((j & (j + 1)) == 0) {  // window of j + 1 = 2^k rows complete
                const int k = 31 - __clz(j + 1);
                const bool kept = scheme == 0 || (k & 1) == 0;
                const int slot = scheme == 0 ? k : k / 2;
                if (kept && i + (1u << k) <= n)
                    reinterpret_cast<uint4 *>(tab + ((uint64_t)slot * n + i) * S)[c] = acc;
            }
        }
    }
}

// Correctly rounded (to nearest, ties to even) conversion of hi*2^64 + lo to
// double: shift the value into 64 bits keeping a sticky bit for everything
// shifted out, let the hardware round the 64-bit integer, scale back exactly.
__device__ __forceinline__ double u128_to_double(uint64_t hi, uint64_t lo) {
    if (hi == 0) return __ull2double_rn(lo);
    const int k = 64 - __clzll((long long)hi);  // significant bits in hi, 1..64
    uint64_t y, sticky;
    if (k == 64) {
        y = hi;
        sticky = lo != 0;
    } else {
        y = (hi << (64 - k)) | (lo >> k);
        sticky = (lo & ((1ull << k) - 1ull)) != 0;
    }
    const double scale = __longlong_as_double((long long)(1023 + k) << 52);  // 2^k
    return __dmul_rn(__ull2double_rn(y | sticky), scale);
}

// Exact integer part of the HLL harmonic sum over register bytes
// [b0, b1) of node v (slice-major storage whose slice 0 holds byte b0 ... of
// every node): lo/hi accumulate sum of 2^(K - M) over the registers M >= 1,
// zeros counts M = 0 (K = 65 - p).  Warp-cooperative; every lane ends with the
// warp's totals.
__device__ __forceinline__ void harmonic_partial(const uint8_t *__restrict__ regs, uint32_t n, int p, int S,
                                                 uint32_t b0, uint32_t b1, uint32_t v, int lane, bool nib,
                                                 uint64_t &lo, uint64_t &hi, uint32_t &zeros) {
    const int K = 65 - p;
    lo = 0;
    hi = 0;
    zeros = 0;
    const int fields = nib ? 8 : 4;  // registers per 32-bit word
    const int width = nib ? 4 : 8;
    const uint32_t fmask = nib ? 0xFu : 0xFFu;
    for (uint32_t r0 = b0 + (uint32_t)lane * 16u; r0 < b1; r0 += 32u * 16u) {
        const uint32_t rel = r0 - b0;
        const uint32_t s = rel / (uint32_t)S, o = rel % (uint32_t)S;
        const uint4 x = *reinterpret_cast<const uint4 *>(regs + ((uint64_t)s * n + v) * (uint64_t)S + o);
        const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
        // A lane adds at most m / 32 terms of at most 2^(K-1) = 2^(64-p) each in
        // this loop, so its sum stays below 2^59: no carry into hi here.
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int b = 0; b < fields; b++) {
                const uint32_t M = (wv[i] >> (width * b)) & fmask;
                zeros += M == 0u ? 1u : 0u;
                lo += M == 0u ? 0ull : 1ull << (K - (int)M);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
        const uint64_t olo = __shfl_xor_sync(0xffffffffu, lo, o);
        const uint64_t ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        lo += olo;
        hi += ohi + (lo < olo);
    }
}

// HLL estimator (Sec. 2.3, Sec. 3.3) from the exact harmonic sum, then
// Eq. sumD.  Z = sum_j 2^-M[j] is formed exactly as the integer Z * 2^(65-p)
// (the zero registers' V * 2^(65-p) plus the partial sum lo/hi of
// harmonic_partial) and rounded once, so the result does not depend on
// summation order.  E = alpha_m m^2 / Z; c = lc[V] = m ln(m/V) if E <= 2.5m
// and V > 0, else E.  For t >= 1: sum_d += t * (c - c_prev), and inc_flag
// records max_v(c - c_prev) > 0.5 (the paper's convergence test).
__device__ __forceinline__ void estimate_finish(uint64_t lo, uint64_t hi, uint32_t zeros, int p, int t,
                                                double alpha_mm, const double *__restrict__ lc,
                                                const double *__restrict__ c_prev, double *__restrict__ c_cur,
                                                double *__restrict__ sum_d, uint32_t *__restrict__ inc_flag,
                                                uint32_t v) {
    const uint32_t m = 1u << p;
    const int K = 65 - p;
    // add V * 2^K (V <= 2^16, K <= 61: fits in 128 bits)
    const uint64_t zlo = (uint64_t)zeros << K;
    const uint64_t zhi = (uint64_t)zeros >> (64 - K);
    lo += zlo;
    hi += zhi + (lo < zlo);
    const double inv_scale = __longlong_as_double((long long)(1023 - K) << 52);  // 2^-K
    const double Z = __dmul_rn(u128_to_double(hi, lo), inv_scale);
    const double E = __ddiv_rn(alpha_mm, Z);
    const double c = (E <= 2.5 * (double)m && zeros > 0) ? lc[zeros] : E;
    if (t > 0) {
        const double diff = __dsub_rn(c, c_prev[v]);
        sum_d[v] = __dadd_rn(sum_d[v], __dmul_rn((double)t, diff));
        if (diff > 0.5 && *reinterpret_cast<volatile uint32_t *>(inc_flag) == 0u) atomicOr(inc_flag, 1u);
    }
    c_cur[v] = c;
}

// Estimator and Eq. sumD for node v over all its registers (one warp; lane 0
// writes the results).
__device__ __forceinline__ void estimate_node(const uint8_t *__restrict__ regs, uint32_t n, int p, int S, int t,
                                              double alpha_mm, const double *__restrict__ lc,
                                              const double *__restrict__ c_prev, double *__restrict__ c_cur,
                                              double *__restrict__ sum_d, uint32_t *__restrict__ inc_flag, uint32_t v,
                                              int lane, bool nib = false) {
    const uint32_t node_bytes = nib ? (1u << p) / 2u : (1u << p);  // 4-bit registers: two per byte
    uint64_t lo, hi;
    uint32_t zeros;
    harmonic_partial(regs, n, p, S, 0u, node_bytes, v, lane, nib, lo, hi, zeros);
    if (lane != 0) return;
    estimate_finish(lo, hi, zeros, p, t, alpha_mm, lc, c_prev, c_cur, sum_d, inc_flag, v);
}

// MD(v) = sum_d[v] / (N_v - 1) (Sec. 3.3), NaN when N_v <= 1; ball = c_t.
__device__ __forceinline__ void finalize_node(uint32_t n, const uint32_t *__restrict__ comp,
                                              const double *__restrict__ sum_d, const double *__restrict__ c,
                                              double *__restrict__ md, double *__restrict__ ball, uint32_t v) {
    const double nv = comp ? (double)comp[v] : (double)n;
    if (md) md[v] = (nv <= 1.0) ? __longlong_as_double(0x7FF8000000000000ll) : __ddiv_rn(sum_d[v], __dsub_rn(nv, 1.0));
    if (ball) ball[v] = c[v];
}

}  // namespace
}  // namespace vga
