// hyperball.cu -- HyperBall (Algorithm 1, Sec. 3.3) on the device-resident
// compressed CSR: counter initialisation, the register-wise union of
// Eq. hll-union (per run of consecutive neighbour ids through a per-slice
// table of range maxima, or per neighbour with on-the-fly LEB128 decoding),
// the HLL estimator, the distance accumulation of Eq. sumD and Visual Mean
// Depth; plus the register-range shards of one analysis.
//
// Register layout: the N x m uint8 registers are stored slice-major,
// [m/S][N][S] for a slice width of S bytes, so that one union launch touches
// only N*S bytes of counters (the slice and its table sized to stay resident
// in L2) and every gather is S contiguous, 16-byte aligned bytes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "hb_device.cuh"

namespace vga {

// HLL alpha_m (Flajolet et al. 2007).
double hll_alpha_host(int p) {
    const double m = (double)(1u << p);
    if (p == 4) return 0.673;
    if (p == 5) return 0.697;
    if (p == 6) return 0.709;
    return 0.7213 / (1.0 + 1.079 / m);
}

// Linear-counting table m ln(m / V), V = 1..m, computed once per p on the host
// so that the device and any host consumer see the same doubles.
const std::vector<double> &lc_table(int p) {
    static std::vector<double> tables[17];
    static bool ready[17] = {false};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[p]) {
        const uint32_t m = 1u << p;
        std::vector<double> t(m + 1, 0.0);
        for (uint32_t V = 1; V <= m; V++) t[V] = (double)m * std::log((double)m / (double)V);
        tables[p].swap(t);
        ready[p] = true;
    }
    return tables[p];
}

namespace {

// Alg. 1 initialisation; with `keys` given, each node's key for the first
// pass's scatter as well (KeyFmt: 16-bit for p <= kKey16MaxP, else 32-bit).
__global__ void hb_init_kernel(uint8_t *__restrict__ regs, uint32_t n, int p, int S, uint64_t seed, int nib,
                               uint32_t s0, uint32_t s1, void *__restrict__ keys) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    init_node(regs, n, p, S, seed, (uint32_t)v, nib != 0, s0, s1);
    if (keys) {
        const uint32_t key = node_key((uint32_t)v, p, seed, nib != 0);
        if (p <= kKey16MaxP)
            static_cast<uint16_t *>(keys)[v] = KeyFmt<uint16_t>::pack(key);
        else
            static_cast<uint32_t *>(keys)[v] = KeyFmt<uint32_t>::pack(key);
    }
}

// First pass of the per-neighbour variant as a scatter (first_pass_csr), one
// warp per node; each warp holds m words of shared memory (its register cells).
template <bool NIB, class K>
__global__ void __launch_bounds__(128) hb_first_pass_csr_kernel(const uint64_t *__restrict__ off,
                                                                const uint8_t *__restrict__ bytes,
                                                                const K *__restrict__ keys, uint32_t n, int p,
                                                                int s_log2, uint32_t s0, uint32_t s1,
                                                                uint8_t *__restrict__ nxt,
                                                                uint32_t *__restrict__ flags,
                                                                uint8_t *__restrict__ chg) {
    extern __shared__ __align__(16) uint32_t s_cells[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n) return;
    const uint32_t m = 1u << p;
    first_pass_csr<NIB, K>(off, bytes, keys, (uint32_t)warp, n, p, s_log2, s0, s1, nxt,
                           s_cells + (uint64_t)wib * m, lane, flags, reinterpret_cast<int *>(flags + 2), chg);
}

// First pass of Eq. hll-union as a scatter of the nodes' keys (first_pass_item),
// one warp per work item; all slices in one launch.  Each warp holds m + 32
// words of shared memory (its register cells, then its lookup stage).
template <bool NIB, class K>
__global__ void __launch_bounds__(128) hb_first_pass_kernel(const RunItem *__restrict__ items, uint64_t n_items,
                                                            const uint32_t *__restrict__ lk,
                                                            const K *__restrict__ keys, uint32_t n, int p,
                                                            int scheme, int s_log2, uint32_t s0, uint32_t s1,
                                                            uint8_t *__restrict__ nxt, uint32_t *__restrict__ flags,
                                                            uint8_t *__restrict__ chg) {
    extern __shared__ __align__(16) uint32_t s_cells[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n_items) return;
    const uint32_t m = 1u << p;
    uint32_t *cells = s_cells + (uint64_t)wib * (m + 32u);
    first_pass_item<NIB, K>(items[warp], lk, keys, n, p, scheme, s_log2, s0, s1, nxt, cells, cells + m, lane, flags,
                         reinterpret_cast<int *>(flags + 2), chg);
}

// Eq. hll-union for one register slice, one warp per node (union_node_edges).
template <int S, bool NIB>
__global__ void __launch_bounds__(512) hb_union_kernel(const uint64_t *__restrict__ off,
                                                       const uint8_t *__restrict__ bytes,
                                                       const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt,
                                                       uint32_t n, uint32_t *__restrict__ flags,
                                                       const uint32_t *__restrict__ need, int s,
                                                       uint8_t *__restrict__ chg) {
    extern __shared__ uint32_t s_ids[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n) return;
    if (need && !((need[warp] >> s) & 1u)) {  // a change-tracked pass: no neighbour changed this slice
        keep_item<S, NIB>(cur, nxt, (uint32_t)warp, false, lane, reinterpret_cast<int *>(flags + 2));
        return;
    }
    union_node_edges<S, NIB>(off, bytes, cur, nxt, (uint32_t)warp, s_ids + wib * 32, lane, flags, chg);
}

// Register cap of the run-aware union kernels: 64 registers a thread lets 8
// CTAs of 4 warps share an SM (measured faster than the uncapped ~70 on the
// city workload), and a CTA of up to 1024 threads still launches.
#define VGA_UNION_MAXNREG 64

// Run-aware Eq. hll-union for one register slice, one warp per work item
// (RunItem: a whole node, or one chunk of a split hub), after the slice's
// table region has been built: the item's range lookups stream through the
// warp's TMA stage and each lookup's table row is gathered (lean_fold).
// flags[2] records a bounded wait that ran out.  With need given (a
// change-tracked pass), a node whose bit `s` is clear keeps its registers
// (keep_item); with chg given, changed nodes are recorded in it (the slice's
// change bytes).
template <int S, bool NIB>
__global__ void __maxnreg__(VGA_UNION_MAXNREG) hb_union_runs_kernel(
    const RunItem *__restrict__ items, uint64_t n_items, const uint32_t *__restrict__ lk,
    const uint8_t *__restrict__ cur, const uint8_t *__restrict__ tab, uint8_t *__restrict__ nxt, uint32_t n,
    uint32_t *__restrict__ flags, const uint32_t *__restrict__ need, int s, uint8_t *__restrict__ chg) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp >= n_items) return;
    const RunItem it = items[warp];
    const uint32_t v = it.v & ~kHubChunk;
    const bool hub = (it.v & kHubChunk) != 0;
    int *err = reinterpret_cast<int *>(flags + 2);
    if (need && !((need[v] >> s) & 1u)) {
        keep_item<S, NIB>(cur, nxt, v, hub, lane, err);
        return;
    }
    LkStage &st = reinterpret_cast<LkStage *>(s_dyn)[wib];
    lk_stage_init(st, lane);
    uint32_t phase = 0;
    union_item<S, NIB>(it, lk, cur, tab, nxt, st, phase, lane, flags, err, chg);
}

// Grouped run-aware Eq. hll-union for one register slice, one warp per group
// of NODES consecutive nodes (GroupItem; runs.cu builds the lists): the
// group's distinct rows stream through the warp's TMA stage class by class;
// each class's rows are gathered and folded into one accumulator, which at the
// class's end is reduced over the warp and max-merged into the shared-memory
// partial rows of the class's nodes.  Finally every node's partial is maxed
// with its own registers and stored (lean_store).  The maximum over each
// node's rows is that over its own lookup list, so the registers equal those
// of hb_union_runs_kernel bit for bit.  With need given, a group none of whose
// nodes needs slice `s` keeps its registers; otherwise all its nodes are
// recomputed (a node that needed nothing gets its own registers back).
// Shared memory per warp: an LkStage, then NODES rows of S bytes.
template <int S, bool NIB, int NODES>
__global__ void __maxnreg__(VGA_UNION_MAXNREG) hb_union_groups_kernel(
    const GroupItem *__restrict__ items, uint64_t n_items, const uint32_t *__restrict__ rows,
    const uint2 *__restrict__ cls, const uint8_t *__restrict__ cur, const uint8_t *__restrict__ tab,
    uint8_t *__restrict__ nxt, uint32_t *__restrict__ flags, const uint32_t *__restrict__ need, int s,
    uint8_t *__restrict__ chg) {
    constexpr int W16 = S / 16;  // uint4 words of a slice row
    extern __shared__ __align__(128) unsigned char s_dyn[];
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    LkStage &st = reinterpret_cast<LkStage *>(s_dyn)[wib];
    uint4 *part = reinterpret_cast<uint4 *>(s_dyn + (size_t)nw * sizeof(LkStage)) + (size_t)wib * NODES * W16;
    const uint64_t warp = (uint64_t)blockIdx.x * nw + wib;
    if (warp >= n_items) return;
    const GroupItem &gi = items[warp];  // node ids are read again where needed, not held in registers
    int *err = reinterpret_cast<int *>(flags + 2);
    if (need) {
        bool any = false;
#pragma unroll
        for (int j = 0; j < NODES; j++) {
            const uint32_t v = gi.node[j];
            any |= v != 0xffffffffu && ((need[v] >> s) & 1u);
        }
        if (!any) {
#pragma unroll
            for (int j = 0; j < NODES; j++) {
                const uint32_t v = gi.node[j];
                if (v != 0xffffffffu) keep_item<S, NIB>(cur, nxt, v, false, lane, err);
            }
            return;
        }
    }
    lk_stage_init(st, lane);
    uint32_t phase = 0;
    union_group<S, NIB, NODES>(gi, rows, cls, cur, tab, nxt, part, st, phase, lane, flags, err, chg);
}

// Change-tracked passes.  The union of pass t records, per slice s, which nodes
// changed (change bytes chg[s][v], 0 or 1).  A later pass t + 1 needs to
// recompute node v in slice s only if some neighbour of v changed slice s in
// pass t; hb_ortab_kernel and hb_need_kernel find those nodes through the
// run-aware union's own range lookups.

// Number of (node, slice) pairs that changed in the pass just run: the change
// bytes are 0 or 1, so the set bits of each 32-bit word count them.
__global__ void hb_count_kernel(const uint32_t *__restrict__ words, uint64_t n_words,
                                unsigned long long *__restrict__ count) {
    __shared__ uint32_t part[32];
    uint32_t c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words;
         i += (uint64_t)gridDim.x * blockDim.x)
        c += __popc(words[i]);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        if (t) atomicAdd(count, t);
    }
}

// Range-OR table of the change masks: row r = slot * n + i holds, bit s per
// slice, whether a node of the window [i, i + w) changed slice s, w being the
// window width of the slot in the table scheme (the rows and row indices of
// the table of range maxima, so that a range lookup addresses both).
// `rows` rows of the scheme are built (1: the per-node masks alone, which the
// per-neighbour variant ORs over decoded ids).
__global__ void hb_ortab_kernel(const uint8_t *__restrict__ chg, uint32_t n, int slices, int scheme, int rows,
                                uint32_t *__restrict__ ortab) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t acc = 0;
    int slot = 0;
    for (uint32_t j = 0; j < (1u << kRunLevels) && slot < rows; j++) {
        if (i + j < n)
            for (int sl = 0; sl < slices; sl++) acc |= (uint32_t)chg[(uint64_t)sl * n + i + j] << sl;
        const int level = scheme == 0 ? slot : 2 * slot;
        if (j + 1u == (1u << level)) ortab[(uint64_t)slot++ * n + i] = acc;
    }
}

// need[v], bit s: one of node v's range lookups covers a node that changed
// slice s in the previous pass.  One warp per work item; split hubs OR their
// chunks' masks together (need is zeroed first).  A warp stops early once
// every slice is needed.
__global__ void __launch_bounds__(256) hb_need_kernel(const RunItem *__restrict__ items, uint64_t n_items,
                                                      const uint32_t *__restrict__ lk,
                                                      const uint32_t *__restrict__ ortab, uint32_t all,
                                                      uint32_t *__restrict__ need) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= n_items) return;
    const RunItem it = items[warp];
    const uint64_t e = it.b + it.cnt;
    uint32_t acc = 0;
    uint64_t kb = it.b;  // whole chunks of 256 lookups first (a warp-uniform loop)
    for (; kb + 256u <= e; kb += 256u) {
        uint32_t r[8];
#pragma unroll
        for (int u = 0; u < 8; u++) r[u] = __ldcs(lk + kb + u * 32u + lane);
#pragma unroll
        for (int u = 0; u < 8; u++) acc |= __ldg(ortab + r[u]);
        if (__reduce_or_sync(0xffffffffu, acc) == all) break;
    }
    if (__reduce_or_sync(0xffffffffu, acc) != all)
        for (uint64_t k = kb + lane; k < e; k += 32u) acc |= __ldg(ortab + __ldcs(lk + k));
    acc = __reduce_or_sync(0xffffffffu, acc);
    if (lane == 0) {
        if (it.v & kHubChunk)
            atomicOr(need + (it.v & ~kHubChunk), acc);
        else
            need[it.v] = acc;
    }
}

// need[v] for the per-neighbour variant: the warp decodes node v's list
// (decode_window) and ORs the change masks (`masks`, one u32 per node) of the
// decoded ids, stopping once every slice is needed.
__global__ void __launch_bounds__(256) hb_need_csr_kernel(const uint64_t *__restrict__ off,
                                                          const uint8_t *__restrict__ bytes, uint32_t n,
                                                          const uint32_t *__restrict__ masks, uint32_t all,
                                                          uint32_t *__restrict__ need) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= n) return;
    uint64_t pos = off[warp];
    const uint64_t end = off[warp + 1];
    uint32_t base = 0, acc = 0;
    while (pos < end) {
        const WindowDecode<uint32_t> r = decode_window<uint32_t>(bytes, pos, end, base, lane);
        if (r.term_mask == 0) break;  // cannot happen on a validated graph; guarantees progress
        if ((r.term_mask >> lane) & 1u) acc |= __ldg(masks + r.id);
        if (__reduce_or_sync(0xffffffffu, acc) == all) break;
        base = r.next_base;
        pos += (uint64_t)r.advance;
    }
    acc = __reduce_or_sync(0xffffffffu, acc);
    if (lane == 0) need[warp] = acc;
}

// The slice's table region (table_item: T_0 and the scheme's levels), B rows
// per CTA of 256 threads, in one launch.
template <int S, bool NIB>
__global__ void __launch_bounds__(256) hb_table_kernel(const uint8_t *__restrict__ cur, uint8_t *__restrict__ tab,
                                                       uint32_t n, int scheme) {
    __shared__ __align__(16) uint8_t buf[TableShape<S>::R * S];
    table_item<S, NIB>(cur, tab, n, blockIdx.x * (uint32_t)TableShape<S>::B, buf, scheme);
}

// Microbenchmark twin of hb_union_kernel: rows drawn from a hash instead of
// decoded from the CSR.  XOR = false folds them with the union's gather_fold
// (the union loop's own ceiling); XOR = true only xors the loaded words, which
// leaves the gathers themselves as the limit (the L2 gather bandwidth).
template <int S, bool XOR>
__global__ void __launch_bounds__(512) gather_bench_kernel(const uint8_t *__restrict__ buf, uint32_t rows,
                                                           uint32_t windows, uint32_t *__restrict__ out) {
    using Sh = GatherShape<S>;
    extern __shared__ uint32_t s_ids[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *ids = s_ids + wib * 32;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int g = lane / Sh::G, sub = lane % Sh::G;
    RegFmt<false>::Acc acc[4 * Sh::V4] = {};
    uint32_t x_acc = 0;
    for (uint32_t w = 0; w < windows; w++) {
        ids[lane] = (uint32_t)(splitmix64((warp * windows + w) * 32 + lane) % rows);
        __syncwarp();
        if (XOR) {
            for (int k0 = 0; k0 < 32; k0 += Sh::P * Sh::U) {
                uint4 x[Sh::U][Sh::V4];
#pragma unroll
                for (int u = 0; u < Sh::U; u++) {
                    const int k = k0 + u * Sh::P + g;
                    if (k < 32) {
                        load_row_chunk<Sh::V4>(buf + (uint64_t)ids[k] * S + sub * Sh::CH, x[u]);
                    } else {
#pragma unroll
                        for (int q = 0; q < Sh::V4; q++) x[u][q] = make_uint4(0, 0, 0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < Sh::U; u++)
#pragma unroll
                    for (int q = 0; q < Sh::V4; q++) x_acc ^= x[u][q].x ^ x[u][q].y ^ x[u][q].z ^ x[u][q].w;
            }
        } else {
            gather_fold<S, false>(SliceRow<S>{buf}, ids, 32, g, sub, acc);
        }
        __syncwarp();
    }
    if (!XOR) {
        uint4 r[Sh::V4];
        finish_groups<S, false>(acc, r);
        x_acc = r[0].x ^ r[0].y ^ r[0].z ^ r[0].w;
    }
    if (lane == 0) out[warp] = x_acc;
}

// Shape-independent L2 read ceiling: every thread streams 16-byte words of an
// L2-resident buffer, consecutive threads on consecutive words (whole 128-byte
// lines per 8 lanes), grid-stride, R passes over the buffer, 8 loads in flight
// per thread, cached in L2 only (ld.global.cg) so that L1 hits cannot inflate
// the figure.  The loaded words are xored into one word per warp.
__global__ void __launch_bounds__(512) stream_bench_kernel(const uint4 *__restrict__ buf, uint64_t words,
                                                           uint32_t passes, uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t r = 0; r < passes; r++) {
        uint64_t i = t0;
        for (; i + 7 * stride < words; i += 8 * stride) {
            uint4 x[8];
#pragma unroll
            for (int u = 0; u < 8; u++) x[u] = __ldcg(buf + i + u * stride);
#pragma unroll
            for (int u = 0; u < 8; u++) acc ^= x[u].x ^ x[u].y ^ x[u].z ^ x[u].w;
        }
        for (; i < words; i += stride) {
            const uint4 x = __ldcg(buf + i);
            acc ^= x.x ^ x.y ^ x.z ^ x.w;
        }
    }
    acc = __reduce_xor_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0) out[t0 >> 5] = acc;
}

// HLL estimate of every node, then Eq. sumD (estimate_node); flags[1]
// records the paper's convergence test max_v(c_t - c_{t-1}) > 0.5.
__global__ void hb_estimate_kernel(const uint8_t *__restrict__ regs, uint32_t n, int p, int S, int t,
                                   double alpha_mm, const double *__restrict__ lc, const double *__restrict__ c_prev,
                                   double *__restrict__ c_cur, double *__restrict__ sum_d,
                                   uint32_t *__restrict__ flags, int nib) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= n) return;
    estimate_node(regs, n, p, S, t, alpha_mm, lc, c_prev, c_cur, sum_d, flags + 1, (uint32_t)warp, lane, nib != 0);
}

// Register-range shard: node v's exact partial harmonic sum over the shard's
// slices (relative slice 0 = register byte s0 * S) and its zero count, into
// the shard's partial block (u64 sums, then u32 counts).  A shard holds fewer
// than m registers, so the sum stays below 2^64; flags[2] would record
// otherwise.
__global__ void hb_shard_partial_kernel(const uint8_t *__restrict__ regs, uint32_t n, int p, int S, uint32_t b0,
                                        uint32_t b1, int nib, uint64_t *__restrict__ part_sum,
                                        uint32_t *__restrict__ part_zeros, uint32_t *__restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= n) return;
    uint64_t lo, hi;
    uint32_t zeros;
    harmonic_partial(regs, n, p, S, b0, b1, (uint32_t)warp, lane, nib != 0, lo, hi, zeros);
    if (lane != 0) return;
    if (hi) atomicOr(flags + 2, 2u);
    part_sum[warp] = lo;
    part_zeros[warp] = zeros;
}

// Estimator and Eq. sumD from all shards' partial blocks (`blocks` of
// `block_bytes` each, in shard order): the partial sums are added exactly in
// 128 bits, the zero counts as integers, so every shard count gives the
// unsharded result bit for bit.  One thread per node.
__global__ void hb_shard_estimate_kernel(const uint8_t *__restrict__ parts, int blocks, uint64_t block_bytes,
                                         uint64_t zeros_off, uint32_t n, int p, int t, double alpha_mm,
                                         const double *__restrict__ lc, const double *__restrict__ c_prev,
                                         double *__restrict__ c_cur, double *__restrict__ sum_d,
                                         uint32_t *__restrict__ flags) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint64_t lo = 0, hi = 0;
    uint32_t zeros = 0;
    for (int b = 0; b < blocks; b++) {
        const uint8_t *blk = parts + (uint64_t)b * block_bytes;
        const uint64_t x = reinterpret_cast<const uint64_t *>(blk)[v];
        lo += x;
        hi += (lo < x);
        zeros += reinterpret_cast<const uint32_t *>(blk + zeros_off)[v];
    }
    estimate_finish(lo, hi, zeros, p, t, alpha_mm, lc, c_prev, c_cur, sum_d, flags + 1, (uint32_t)v);
}

// MD(v) = sum_d[v] / (N_v - 1) (Sec. 3.3), NaN when N_v <= 1; ball = c_t.
__global__ void hb_finalize_kernel(uint32_t n, const uint32_t *__restrict__ comp, const double *__restrict__ sum_d,
                                   const double *__restrict__ c, double *__restrict__ md, double *__restrict__ ball) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    finalize_node(n, comp, sum_d, c, md, ball, (uint32_t)v);
}


// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

constexpr int kModePerEdge = 1;  // one gather per neighbour (hb_union_kernel)
constexpr int kModeRuns = 2;     // one or two gathers per run of consecutive ids (hb_union_runs_kernel)

struct Plan {
    int p = 10;
    uint32_t m = 1024;
    int nib = 0;           // 4-bit registers, two per byte (the paper's packed format)
    uint32_t node_bytes = 1024;  // register bytes per node: m, or m / 2 with 4-bit registers
    int S = 1024;          // slice bytes
    int slices = 1;
    int warps = 8;         // union kernel warps per CTA
    int mode = kModeRuns;  // union variant
    int scheme = 0;        // runs mode: table scheme (table_rows(scheme) rows per node and slice)
    uint32_t hub_req = 0;  // runs mode: requested hub threshold (0 = automatic)
    uint32_t hub = 0;      // runs mode: nodes with more lookups than this are split across warps
    RunItemList items;     // runs mode: the union's work list for `hub`
    int group = 0;         // runs mode: nodes per group of the grouped union (0: one node per warp)
    GroupList groups;      // runs mode with group > 0: the grouped lookup lists for `hub`
    bool first_scatter = false;  // pass 1 by the scatter of the nodes' keys (kept at off_tab)
    int track = 0;               // runs mode, slices <= 32: change tracking (0 off, 1 automatic, 2 every pass)
    uint64_t n = 0;
    // workspace layout (byte offsets, 256-aligned)
    uint64_t off_cur = 0, off_next = 0, off_c0 = 0, off_c1 = 0, off_sum = 0, off_lc = 0, off_flags = 0, off_tab = 0,
             off_chg = 0, off_need = 0, off_ortab = 0, chg_bytes = 0, total = 0;
};

static uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Group size of the grouped run-aware union when the caller leaves it open:
// four consecutive nodes (measured fastest of 2, 4 and 8 on the city graph).
constexpr int kGroupAutoNodes = 4;

// Change tracking keeps one bit per slice in a 32-bit mask per node.
constexpr int kTrackMaxSlices = 32;
// The automatic rule tracks a pass when the previous one changed fewer than
// this share of the (node, slice) pairs: after a pass that changed more,
// nearly every node has a changed neighbour in every slice.
constexpr double kTrackBelow = 0.01;


// Hub threshold of the run-aware union (lookups per work item).
static uint32_t hub_threshold(const vga_graph *g, int scheme, uint32_t requested) {
    return requested > 0 ? requested : hub_lookups_auto(g, scheme);
}

static int make_plan(const vga_graph *g, int p, const vga_tuning *tune, Plan *P) {
    if (p < 4 || p > 16) {
        set_error("precision p = %d is outside 4..16", p);
        return VGA_EINVAL;
    }
    P->p = p;
    P->m = 1u << p;
    P->n = g->n;
    const int bits = tune && tune->register_bits ? tune->register_bits : 8;
    if (bits != 8 && bits != 4) {
        set_error("register_bits = %d must be 8 or 4", bits);
        return VGA_EINVAL;
    }
    if (bits == 4 && p < 5) {
        set_error("4-bit registers need p >= 5 (got %d)", p);
        return VGA_EINVAL;
    }
    P->nib = bits == 4;
    P->node_bytes = P->nib ? P->m / 2 : P->m;
    // fields left at 0 come from the autotuner's table entry for the graph's
    // degree bucket, if one is installed, else from the built-in defaults
    vga_tune_entry te{};
    const bool tabled = tune_table_lookup(g, &te);
    const int req_mode = (tune && tune->union_mode) ? tune->union_mode : 0;
    if (req_mode < 0 || req_mode > kModeRuns) {
        set_error("union_mode = %d must be 0 (auto), 1 (per neighbour) or 2 (per run)", req_mode);
        return VGA_EINVAL;
    }
    if (req_mode == kModeRuns && (uint64_t)g->n > kRunMaxNodes) {
        set_error("union_mode 2 supports at most 2^29 nodes (graph has %u)", g->n);
        return VGA_EINVAL;
    }
    const bool runs_ok = (uint64_t)g->n <= kRunMaxNodes;
    P->mode = req_mode ? req_mode
                       : (tabled && te.union_mode == kModePerEdge) || !runs_ok ? kModePerEdge : kModeRuns;
    // table scheme (runs mode): the graph's own unless the caller asks for one
    const int levels = tune ? tune->table_levels : 0;
    if (levels != 0 && levels != 5 && levels != 3) {
        set_error("table_levels = %d must be 0 (automatic), 5 or 3", levels);
        return VGA_EINVAL;
    }
    P->scheme = levels == 5 ? 0 : levels == 3 ? 1 : g->lk_scheme;
    // grouped union (runs mode): nodes per group, 0 for one node per warp
    const int grp = tune ? tune->group_nodes : 0;
    if (grp != 0 && grp != 1 && grp != 2 && grp != 4 && grp != 8) {
        set_error("group_nodes = %d must be 0 (automatic), 1 (one node per warp), 2, 4 or 8", grp);
        return VGA_EINVAL;
    }
    const int grp_sel = grp ? grp : (tabled && te.group_nodes > 0) ? te.group_nodes : 0;
    P->group = P->mode != kModeRuns || grp_sel == 1 ? 0 : grp_sel == 0 ? kGroupAutoNodes : grp_sel;
    // rows of counters the union reads per slice: the slice, or in runs mode its table region
    const uint64_t rows_per_node = P->mode == kModeRuns ? (uint64_t)table_rows(P->scheme) : 1;
    int S = tune ? tune->slice_bytes : 0;
    if (S != 0) {
        if (S < 16 || S > 1024 || (S & (S - 1)) || (uint32_t)S > P->node_bytes) {
            set_error("slice_bytes = %d must be a power of two in [16, min(register bytes per node, 1024)]", S);
            return VGA_EINVAL;
        }
    } else {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device);
        const uint64_t l2_bytes = (uint64_t)(l2 > 0 ? l2 : (64 << 20));
        // a tabled width is an upper bound; the slice must still fit the whole L2
        const bool tabled_S = tabled && te.slice_bytes > 0 && !(tune && tune->l2_budget_mb > 0);
        uint64_t budget = (tune && tune->l2_budget_mb > 0) ? (uint64_t)tune->l2_budget_mb << 20
                          : tabled_S                       ? l2_bytes
                          : P->mode == kModeRuns && P->group ? grouped_l2_budget(g->device)
                          : P->mode == kModeRuns           ? union_l2_budget(g->device)
                                                           : l2_bytes * 6 / 10;
        S = (int)std::min<uint32_t>(P->node_bytes, tabled_S ? (uint32_t)std::min(te.slice_bytes, 1024) : 1024u);
        while (S > 16 && (uint64_t)S * P->n * rows_per_node > budget) S >>= 1;
    }
    P->S = S;
    P->slices = (int)(P->node_bytes / (uint32_t)S);
    // default CTA size: 4 warps for the run-aware union (measured fastest on
    // the city workload), 8 for the per-neighbour one
    P->warps = (tune && tune->warps_per_cta > 0) ? tune->warps_per_cta
               : (tabled && te.warps_per_cta > 0)     ? te.warps_per_cta
               : P->mode == kModeRuns                 ? 4
                                                      : 8;
    if (P->warps > 16) {
        set_error("warps_per_cta = %d exceeds 16", P->warps);
        return VGA_EINVAL;
    }
    if (tune && tune->hub_lookups < 0) {
        set_error("hub_lookups = %d must be >= 0", tune->hub_lookups);
        return VGA_EINVAL;
    }
    P->hub_req = (tune && tune->hub_lookups > 0) ? (uint32_t)tune->hub_lookups
                 : (tabled && te.hub_lookups > 0) ? (uint32_t)te.hub_lookups
                                                  : 0u;
    const int first = tune ? tune->first_pass : 0;
    if (first < 0 || first > 2) {
        set_error("first_pass = %d must be 0 (automatic), 1 (gather) or 2 (scatter)", first);
        return VGA_EINVAL;
    }
    const bool scatter_ok = p <= kFirstPassMaxP;
    if (first == 2 && !scatter_ok) {
        set_error("first_pass = 2 (scatter) needs p <= %d", kFirstPassMaxP);
        return VGA_EINVAL;
    }
    P->first_scatter = scatter_ok && first != 1;
    const uint64_t regs = (uint64_t)P->n * P->node_bytes;
    uint64_t o = 0;
    P->off_cur = o;   o = align256(o + regs);
    P->off_next = o;  o = align256(o + regs);
    P->off_c0 = o;    o = align256(o + 8 * P->n);
    P->off_c1 = o;    o = align256(o + 8 * P->n);
    P->off_sum = o;   o = align256(o + 8 * P->n);
    P->off_lc = o;    o = align256(o + 8 * ((uint64_t)P->m + 1));
    P->off_flags = o; o = align256(o + 64);
    // the table region; pass 1's scatter keeps the nodes' keys there (mode 1 has
    // no table region otherwise)
    P->off_tab = o;
    if (P->mode == kModeRuns) o = align256(o + (uint64_t)table_rows(P->scheme) * P->n * (uint64_t)S);
    else if (P->first_scatter) o = align256(o + 4 * P->n);
    const int track = tune ? tune->track_changes : 0;
    if (track < 0 || track > 2) {
        set_error("track_changes = %d must be 0 (automatic), 1 (off) or 2 (every pass)", track);
        return VGA_EINVAL;
    }
    const bool track_ok = P->slices <= kTrackMaxSlices;
    if (track == 2 && !track_ok) {
        set_error("track_changes = 2 needs at most %d slices (have %d)", kTrackMaxSlices, P->slices);
        return VGA_EINVAL;
    }
    P->track = !track_ok || track == 1 ? 0 : track == 2 ? 2 : 1;
    if (P->track) {
        P->chg_bytes = align256((uint64_t)P->slices * P->n);
        P->off_chg = o;   o = align256(o + P->chg_bytes);
        P->off_need = o;  o = align256(o + 4 * P->n);
        P->off_ortab = o;  // range-OR table (mode 2), or the per-node change masks (mode 1)
        o = align256(o + 4ull * (P->mode == kModeRuns ? table_rows(P->scheme) : 1) * P->n);
    }
    P->total = o;
    return VGA_OK;
}


static std::atomic<uint64_t> g_kernel_launches{0};

// Access-policy window (vga_tuning.l2_window): the union's gather source marked
// persisting in L2 on the run's stream, the persisting set-aside raised to fit;
// both restored when the run ends.  In mode 1 the window covers the first
// register slice of `cur` (the slice a launch gathers from moves every launch,
// so only the first of each pass benefits; mode 2 reuses one table region).
struct L2Window {
    cudaStream_t stream = nullptr;
    size_t old_limit = 0;
    cudaStreamAttrValue old_attr{};
    bool active = false;
    int open(cudaStream_t s, void *base, uint64_t bytes, int device) {
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, device);
        if (max_persist <= 0 || max_window <= 0 || !s) return VGA_OK;  // not supported, or the legacy stream
        VGA_CHECK_CUDA(cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize));
        VGA_CHECK_CUDA(cudaStreamGetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &old_attr));
        const size_t window = (size_t)std::min<uint64_t>(bytes, (uint64_t)max_window);
        const size_t setaside = std::min<size_t>(window, (size_t)max_persist);
        VGA_CHECK_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, setaside));
        cudaStreamAttrValue a{};
        a.accessPolicyWindow.base_ptr = base;
        a.accessPolicyWindow.num_bytes = window;
        a.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)setaside / (double)window);
        a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        VGA_CHECK_CUDA(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a));
        stream = s;
        active = true;
        return VGA_OK;
    }
    ~L2Window() {
        if (!active) return;
        cudaStreamSynchronize(stream);
        cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &old_attr);
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
    }
};

// Benchmark counters (vga_profile_*): union launches are bracketed by CUDA
// events on their stream while profiling is on; the events are read after the
// run's final synchronisation.
struct ProfileState {
    std::mutex mu;
    bool enabled = false;
    vga_profile acc{};
};
static ProfileState &prof() {
    static ProfileState s;
    return s;
}

struct PendingTiming {
    cudaEvent_t start, stop;
    uint64_t edges, gather_bytes, hbm_bytes;
    int S, mode, rows;
    bool first;    // the first pass's scatter (hb_first_pass_kernel), not a union slice
    bool tracked;  // a union slice of a change-tracked pass (its work depends on the changes)
};

template <int SS, bool NIB>
static void launch_union_slice(const Plan &P, const vga_graph *g, const uint8_t *c, uint8_t *x, uint8_t *tab,
                               uint32_t *flags, cudaStream_t stream, const uint32_t *need, int s, uint8_t *chg) {
    const unsigned blocks = (unsigned)((P.n + P.warps - 1) / P.warps);
    const size_t smem = (size_t)P.warps * 32 * sizeof(uint32_t);
    if (P.mode == kModeRuns) {
        const unsigned item_blocks = (unsigned)((P.items.count + P.warps - 1) / P.warps);
        const unsigned table_blocks = (unsigned)((P.n + TableShape<SS>::B - 1) / TableShape<SS>::B);
        hb_table_kernel<SS, NIB><<<table_blocks, 256, 0, stream>>>(c, tab, (uint32_t)P.n, P.scheme);
        count_launch();
        if (!P.group) {
            hb_union_runs_kernel<SS, NIB><<<item_blocks, P.warps * 32, (size_t)P.warps * sizeof(LkStage), stream>>>(
                P.items.items, P.items.count, g->lk[P.scheme].d_lk, c, tab, x, (uint32_t)P.n, flags, need, s, chg);
        } else {
            // split hubs (the first items of the work list) per node, then the groups
            if (P.items.hub_items) {
                const unsigned hub_blocks = (unsigned)((P.items.hub_items + P.warps - 1) / P.warps);
                hb_union_runs_kernel<SS, NIB><<<hub_blocks, P.warps * 32, (size_t)P.warps * sizeof(LkStage),
                                                stream>>>(P.items.items, P.items.hub_items, g->lk[P.scheme].d_lk, c,
                                                          tab, x, (uint32_t)P.n, flags, need, s, chg);
                count_launch();
            }
            const size_t smem = (size_t)P.warps * (sizeof(LkStage) + (size_t)P.group * SS);
            const unsigned group_blocks = (unsigned)((P.groups.count + P.warps - 1) / P.warps);
            auto launch_groups = [&](auto kernel) {
                if (smem > (48u << 10))
                    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kernel<<<group_blocks, P.warps * 32, smem, stream>>>(P.groups.items, P.groups.count, P.groups.rows,
                                                                     P.groups.cls, c, tab, x, flags, need, s, chg);
            };
            if (group_blocks) {
                if (P.group == 2) launch_groups(hb_union_groups_kernel<SS, NIB, 2>);
                else if (P.group == 4) launch_groups(hb_union_groups_kernel<SS, NIB, 4>);
                else launch_groups(hb_union_groups_kernel<SS, NIB, 8>);
            }
        }
    } else {
        hb_union_kernel<SS, NIB><<<blocks, P.warps * 32, smem, stream>>>(g->d_offsets, g->d_bytes, c, x, (uint32_t)P.n,
                                                                    flags, need, s, chg);
    }
    count_launch();
}

// One pass of the union over every slice.  need (a change-tracked pass) and
// chg (change bytes to record, [slice][N]) may be null.
static int launch_union(const Plan &P, const vga_graph *g, const uint8_t *cur, uint8_t *nxt, uint8_t *tab,
                        uint32_t *flags, cudaStream_t stream, std::vector<PendingTiming> *timings,
                        const uint32_t *need = nullptr, uint8_t *chg = nullptr) {
    const uint64_t slice_bytes = (uint64_t)P.n * P.S;
    for (int s = 0; s < P.slices; s++) {
        const uint8_t *c = cur + (uint64_t)s * slice_bytes;
        uint8_t *x = nxt + (uint64_t)s * slice_bytes;
        uint8_t *cs = chg ? chg + (uint64_t)s * P.n : nullptr;
        PendingTiming pt{};
        if (timings) {
            VGA_CHECK_CUDA(cudaEventCreate(&pt.start));
            VGA_CHECK_CUDA(cudaEventCreate(&pt.stop));
            VGA_CHECK_CUDA(cudaEventRecord(pt.start, stream));
        }
        switch (P.S) {
            case 16: P.nib ? launch_union_slice<16, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<16, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 32: P.nib ? launch_union_slice<32, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<32, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 64: P.nib ? launch_union_slice<64, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<64, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 128: P.nib ? launch_union_slice<128, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<128, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 256: P.nib ? launch_union_slice<256, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<256, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 512: P.nib ? launch_union_slice<512, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<512, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            case 1024: P.nib ? launch_union_slice<1024, true>(P, g, c, x, tab, flags, stream, need, s, cs)
                             : launch_union_slice<1024, false>(P, g, c, x, tab, flags, stream, need, s, cs); break;
            default:
                set_error("internal: slice width %d", P.S);
                return VGA_EINVAL;
        }
        if (timings) {
            VGA_CHECK_CUDA(cudaEventRecord(pt.stop, stream));
            pt.edges = g->n_edges;
            if (P.mode == kModeRuns && P.group) {
                // distinct rows of the groups plus the split hubs' lookups
                pt.gather_bytes = (P.groups.rows_used + P.groups.hub_rows) * (uint64_t)P.S;
                pt.hbm_bytes = 4 * (P.groups.rows_used + P.groups.hub_rows) + 64 * P.groups.count +
                               16 * P.items.hub_items + 2 * P.n * (uint64_t)P.S;
            } else if (P.mode == kModeRuns) {
                pt.gather_bytes = g->lk[P.scheme].total * (uint64_t)P.S;
                pt.hbm_bytes = 4 * g->lk[P.scheme].total + 16 * P.items.count + 2 * P.n * (uint64_t)P.S;
            } else {
                pt.gather_bytes = g->n_edges * (uint64_t)P.S;
                pt.hbm_bytes = g->n_bytes + 8 * (P.n + 1) + 2 * P.n * (uint64_t)P.S;
            }
            pt.S = P.S;
            pt.mode = P.mode;
            pt.rows = P.mode == kModeRuns ? table_rows(P.scheme) : 1;
            pt.tracked = need != nullptr;
            timings->push_back(pt);
        }
    }
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

// First pass of a run (or of a register-range shard holding slices [s0, s1))
// by the scatter of the nodes' keys; `keys` were written by hb_init_kernel.
static int launch_first_pass(const Plan &P, const vga_graph *g, const void *keys, uint8_t *nxt, uint32_t s0,
                             uint32_t s1, uint32_t *flags, cudaStream_t stream, std::vector<PendingTiming> *timings,
                             uint8_t *chg = nullptr) {
    const size_t smem = (size_t)kFirstPassWarps * (P.m + 32u) * 4u;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        const int most = kFirstPassWarps * ((1 << kFirstPassMaxP) + 32) * 4;
        const void *fns[8] = {reinterpret_cast<const void *>(hb_first_pass_kernel<false, uint16_t>),
                              reinterpret_cast<const void *>(hb_first_pass_kernel<false, uint32_t>),
                              reinterpret_cast<const void *>(hb_first_pass_kernel<true, uint16_t>),
                              reinterpret_cast<const void *>(hb_first_pass_kernel<true, uint32_t>),
                              reinterpret_cast<const void *>(hb_first_pass_csr_kernel<false, uint16_t>),
                              reinterpret_cast<const void *>(hb_first_pass_csr_kernel<false, uint32_t>),
                              reinterpret_cast<const void *>(hb_first_pass_csr_kernel<true, uint16_t>),
                              reinterpret_cast<const void *>(hb_first_pass_csr_kernel<true, uint32_t>)};
        for (const void *f : fns)
            if (attr_err == cudaSuccess)
                attr_err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
    VGA_CHECK_CUDA(attr_err);
    PendingTiming pt{};
    if (timings) {
        VGA_CHECK_CUDA(cudaEventCreate(&pt.start));
        VGA_CHECK_CUDA(cudaEventCreate(&pt.stop));
        VGA_CHECK_CUDA(cudaEventRecord(pt.start, stream));
    }
    const bool runs = P.mode == kModeRuns;
    const uint64_t units = runs ? P.items.count : P.n;  // work items, or nodes in mode 1
    const unsigned blocks = (unsigned)((units + kFirstPassWarps - 1) / kFirstPassWarps);
    const int s_log2 = __builtin_ctz((unsigned)P.S);
    const uint32_t *lk = runs ? g->lk[P.scheme].d_lk : nullptr;
    const uint32_t n = (uint32_t)P.n;
    const bool k16 = P.p <= kKey16MaxP;
#define VGA_FP(NIBV, KT)                                                                                            \
    if (runs)                                                                                                       \
        hb_first_pass_kernel<NIBV, KT><<<blocks, kFirstPassWarps * 32, smem, stream>>>(                            \
            P.items.items, P.items.count, lk, static_cast<const KT *>(keys), n, P.p, P.scheme, s_log2, s0, s1, nxt, \
            flags, chg);                                                                                            \
    else                                                                                                            \
        hb_first_pass_csr_kernel<NIBV, KT><<<blocks, kFirstPassWarps * 32, smem, stream>>>(                        \
            g->d_offsets, g->d_bytes, static_cast<const KT *>(keys), n, P.p, s_log2, s0, s1, nxt, flags, chg)
    if (blocks) {
        if (P.nib) {
            if (k16) VGA_FP(true, uint16_t);
            else VGA_FP(true, uint32_t);
        } else {
            if (k16) VGA_FP(false, uint16_t);
            else VGA_FP(false, uint32_t);
        }
        count_launch();
    }
#undef VGA_FP
    VGA_CHECK_CUDA(cudaGetLastError());
    if (timings) {
        VGA_CHECK_CUDA(cudaEventRecord(pt.stop, stream));
        pt.edges = g->n_edges;
        pt.S = P.S;
        pt.mode = P.mode;
        pt.first = true;
        timings->push_back(pt);
    }
    return VGA_OK;
}

// Before a change-tracked pass: the range-OR table of the previous pass's
// change bytes, then each node's need mask (one bit per slice).  Timed with
// the tracked union slices.
static int launch_need(const Plan &P, const vga_graph *g, const uint8_t *chg, uint32_t *ortab, uint32_t *need,
                       cudaStream_t stream, std::vector<PendingTiming> *timings) {
    PendingTiming pt{};
    if (timings) {
        VGA_CHECK_CUDA(cudaEventCreate(&pt.start));
        VGA_CHECK_CUDA(cudaEventCreate(&pt.stop));
        VGA_CHECK_CUDA(cudaEventRecord(pt.start, stream));
    }
    const bool runs = P.mode == kModeRuns;
    hb_ortab_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(
        chg, (uint32_t)P.n, P.slices, P.scheme, runs ? table_rows(P.scheme) : 1, ortab);
    count_launch();
    const uint32_t all = P.slices >= 32 ? 0xffffffffu : (1u << P.slices) - 1u;
    if (runs) {
        VGA_CHECK_CUDA(cudaMemsetAsync(need, 0, 4 * P.n, stream));
        hb_need_kernel<<<(unsigned)((P.items.count + 7) / 8), 256, 0, stream>>>(
            P.items.items, P.items.count, g->lk[P.scheme].d_lk, ortab, all, need);
    } else {
        hb_need_csr_kernel<<<(unsigned)((P.n + 7) / 8), 256, 0, stream>>>(g->d_offsets, g->d_bytes, (uint32_t)P.n,
                                                                          ortab, all, need);
    }
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    if (timings) {
        VGA_CHECK_CUDA(cudaEventRecord(pt.stop, stream));
        pt.tracked = true;
        timings->push_back(pt);
    }
    return VGA_OK;
}

// (node, slice) pairs the pass changed, into the 64-bit counter at flags + 4.
static int launch_count(const Plan &P, const uint8_t *chg, uint32_t *flags, cudaStream_t stream) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t words = P.chg_bytes / 4;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((words + 255) / 256, (uint64_t)std::max(sms, 1) * 4));
    hb_count_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t *>(chg), words,
                                              reinterpret_cast<unsigned long long *>(flags + 4));
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

// Read the union timings of a run: into the profile counters when profiling is
// on, and summed into *sum_ms when it is given.
static void settle_timings(std::vector<PendingTiming> &timings, bool to_profile, double *sum_ms) {
    ProfileState &ps = prof();
    std::lock_guard<std::mutex> lock(ps.mu);
    for (PendingTiming &pt : timings) {
        float ms = 0.f;
        const bool ok = cudaEventElapsedTime(&ms, pt.start, pt.stop) == cudaSuccess;
        if (sum_ms && !ok) *sum_ms = -1.0;
        if (sum_ms && ok && *sum_ms >= 0.0) *sum_ms += ms;
        if (to_profile && ok && pt.first) {
            ps.acc.first_pass_launches++;
            ps.acc.first_pass_ms += ms;
            ps.acc.first_pass_edges += pt.edges;
        } else if (to_profile && ok && pt.tracked) {
            ps.acc.tracked_launches++;
            ps.acc.tracked_ms += ms;
        } else if (to_profile && ok) {
            ps.acc.union_launches++;
            ps.acc.union_ms += ms;
            ps.acc.union_edges += pt.edges;
            ps.acc.union_gather_bytes += pt.gather_bytes;
            ps.acc.union_hbm_bytes += pt.hbm_bytes;
            ps.acc.slice_bytes = pt.S;
            ps.acc.union_mode = pt.mode;
            ps.acc.table_rows = pt.rows;
        }
        cudaEventDestroy(pt.start);
        cudaEventDestroy(pt.stop);
    }
    timings.clear();
}

static int launch_estimate(const Plan &P, const uint8_t *regs, int t, const double *lc, const double *c_prev,
                           double *c_cur, double *sum_d, uint32_t *flags, cudaStream_t stream) {
    const int warps = 8;
    const unsigned blocks = (unsigned)((P.n + warps - 1) / warps);
    const double alpha_mm = hll_alpha_host(P.p) * (double)P.m * (double)P.m;
    hb_estimate_kernel<<<blocks, warps * 32, 0, stream>>>(regs, (uint32_t)P.n, P.p, P.S, t, alpha_mm, lc, c_prev,
                                                          c_cur, sum_d, flags, P.nib);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

// Registers of one pass into the caller's node-major uint8 trace slot.  With
// 4-bit registers the packed slices are copied to a host buffer and unpacked
// (register j of a node is nibble j % 2 of byte j / 2, low nibble first).
static int copy_trace(const Plan &P, const uint8_t *regs, const double *c, int slot, uint8_t *trace_regs,
                      double *trace_c, cudaStream_t stream) {
    if (trace_regs) {
        uint8_t *dst = trace_regs + (uint64_t)slot * P.n * P.m;
        if (!P.nib) {
            for (int s = 0; s < P.slices; s++)
                VGA_CHECK_CUDA(cudaMemcpy2DAsync(dst + (uint64_t)s * P.S, P.m, regs + (uint64_t)s * P.n * P.S, P.S,
                                                 P.S, P.n, cudaMemcpyDeviceToHost, stream));
        } else {
            std::vector<uint8_t> packed((size_t)P.n * P.node_bytes);
            for (int s = 0; s < P.slices; s++)
                VGA_CHECK_CUDA(cudaMemcpy2DAsync(packed.data() + (uint64_t)s * P.S, P.node_bytes,
                                                 regs + (uint64_t)s * P.n * P.S, P.S, P.S, P.n,
                                                 cudaMemcpyDeviceToHost, stream));
            VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
            for (uint64_t v = 0; v < P.n; v++)
                for (uint32_t b = 0; b < P.node_bytes; b++) {
                    const uint8_t x = packed[v * P.node_bytes + b];
                    dst[v * P.m + 2 * b] = x & 0x0Fu;
                    dst[v * P.m + 2 * b + 1] = x >> 4;
                }
        }
    }
    if (trace_c)
        VGA_CHECK_CUDA(cudaMemcpyAsync(trace_c + (uint64_t)slot * P.n, c, 8 * P.n, cudaMemcpyDeviceToHost, stream));
    return VGA_OK;
}

static int run_impl(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *md_dev, double *ball_dev,
                    int *iterations, void *ws, uint64_t ws_bytes, cudaStream_t stream, const vga_tuning *tune,
                    uint8_t *trace_regs, double *trace_c, int max_trace, double *union_ms = nullptr) {
    if (!g) {
        set_error("null graph");
        return VGA_EINVAL;
    }
    if (conv_mode != 0 && conv_mode != 1) {
        set_error("conv_mode = %d must be 0 or 1", conv_mode);
        return VGA_EINVAL;
    }
    Plan P;
    VGA_TRY(make_plan(g, p, tune, &P));
    DeviceBuffer own_ws;
    if (!ws) {
        VGA_TRY(own_ws.alloc(P.total));
        ws = own_ws.ptr;
    } else if (ws_bytes < P.total || (reinterpret_cast<uintptr_t>(ws) & 255u)) {
        set_error("workspace of %llu bytes at %p: need %llu bytes, 256-byte aligned", (unsigned long long)ws_bytes,
                  ws, (unsigned long long)P.total);
        return VGA_EINVAL;
    }
    uint8_t *base = static_cast<uint8_t *>(ws);
    uint8_t *cur = base + P.off_cur;
    uint8_t *nxt = base + P.off_next;
    double *c_prev = reinterpret_cast<double *>(base + P.off_c0);
    double *c_cur = reinterpret_cast<double *>(base + P.off_c1);
    double *sum_d = reinterpret_cast<double *>(base + P.off_sum);
    double *lc = reinterpret_cast<double *>(base + P.off_lc);
    uint32_t *flags = reinterpret_cast<uint32_t *>(base + P.off_flags);
    uint8_t *tab = base + P.off_tab;
    if (P.mode == kModeRuns && P.n > 0) {
        VGA_TRY(ensure_run_lookups(g, P.scheme, stream));
        P.hub = hub_threshold(g, P.scheme, P.hub_req);
        VGA_TRY(ensure_run_items(g, P.scheme, P.hub, stream, &P.items));
        if (P.group) VGA_TRY(ensure_group_list(g, P.scheme, P.hub, P.group, stream, &P.groups));
    }

    bool profiling;
    {
        std::lock_guard<std::mutex> lock(prof().mu);
        profiling = prof().enabled;
    }
    if (union_ms) *union_ms = 0.0;
    const bool timed = profiling || union_ms;
    std::vector<PendingTiming> timings;
    struct Settle {
        std::vector<PendingTiming> &t;
        bool to_profile;
        double *sum;
        ~Settle() { settle_timings(t, to_profile, sum); }
    } settle{timings, profiling, union_ms};
    const std::vector<double> &table = lc_table(p);
    VGA_CHECK_CUDA(cudaMemcpyAsync(lc, table.data(), 8 * table.size(), cudaMemcpyHostToDevice, stream));
    int t = 0;
    if (P.n > 0) {
        VGA_CHECK_CUDA(cudaMemsetAsync(cur, 0, P.n * P.node_bytes, stream));
        // split hubs merge into next[v] by atomic max: it must start below the result
        if (P.items.hubs) VGA_CHECK_CUDA(cudaMemsetAsync(nxt, 0, P.n * P.node_bytes, stream));
        VGA_CHECK_CUDA(cudaMemsetAsync(sum_d, 0, 8 * P.n, stream));
        void *keys = P.first_scatter ? tab : nullptr;  // tab is unused in pass 1
        hb_init_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(cur, (uint32_t)P.n, p, P.S, seed, P.nib, 0u,
                                                                          (uint32_t)P.slices, keys);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        VGA_TRY(launch_estimate(P, cur, 0, lc, nullptr, c_prev, sum_d, flags, stream));  // c_0
        if (max_trace >= 0) VGA_TRY(copy_trace(P, cur, c_prev, 0, trace_regs, trace_c, stream));
        struct {
            uint32_t f[4];        // changed, estimate increase, bounded wait gave up, unused
            uint64_t n_changed;   // (node, slice) pairs changed by the pass (change tracking)
        } h{};
        VGA_CHECK_CUDA(cudaMemsetAsync(flags, 0, sizeof(h), stream));
        L2Window window;
        if (tune && tune->l2_window) {
            // the bytes every union launch gathers from: the table region, or the register slices
            const uint64_t bytes = P.mode == kModeRuns ? (uint64_t)table_rows(P.scheme) * P.n * P.S : P.n * P.S;
            VGA_TRY(window.open(stream, P.mode == kModeRuns ? tab : cur, bytes, g->device));
        }
        // change tracking: every pass records its changes; a pass after one
        // that changed little recomputes only the nodes with a changed neighbour
        uint8_t *chg = P.track ? base + P.off_chg : nullptr;
        uint32_t *need = P.track ? reinterpret_cast<uint32_t *>(base + P.off_need) : nullptr;
        uint32_t *ortab = P.track ? reinterpret_cast<uint32_t *>(base + P.off_ortab) : nullptr;
        uint64_t changed_prev = ~0ull;
        for (t = 1;; t++) {
            VGA_CHECK_CUDA(cudaMemsetAsync(flags, 0, 8, stream));
            const bool tracked = chg && t >= 2 &&
                                 (P.track == 2 || (double)changed_prev < kTrackBelow * (double)P.n * P.slices);
            if (tracked) VGA_TRY(launch_need(P, g, chg, ortab, need, stream, timed ? &timings : nullptr));
            if (chg) {
                VGA_CHECK_CUDA(cudaMemsetAsync(chg, 0, P.chg_bytes, stream));
                VGA_CHECK_CUDA(cudaMemsetAsync(flags + 4, 0, 8, stream));
            }
            if (t == 1 && keys)
                VGA_TRY(launch_first_pass(P, g, keys, nxt, 0u, (uint32_t)P.slices, flags, stream,
                                          timed ? &timings : nullptr, chg));
            else
                VGA_TRY(launch_union(P, g, cur, nxt, tab, flags, stream, timed ? &timings : nullptr,
                                     tracked ? need : nullptr, chg));
            if (chg) VGA_TRY(launch_count(P, chg, flags, stream));
            VGA_TRY(launch_estimate(P, nxt, t, lc, c_prev, c_cur, sum_d, flags, stream));
            if (t <= max_trace) VGA_TRY(copy_trace(P, nxt, c_cur, t, trace_regs, trace_c, stream));
            VGA_CHECK_CUDA(cudaMemcpyAsync(&h, flags, sizeof(h), cudaMemcpyDeviceToHost, stream));
            VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
            if (h.f[2]) {
                set_error("a bounded wait for a TMA copy ran out in pass %d", t);
                return VGA_ETIMEOUT;
            }
            changed_prev = h.n_changed;
            std::swap(cur, nxt);
            std::swap(c_prev, c_cur);
            const bool stop = (conv_mode == 1) ? (h.f[1] == 0) : (h.f[0] == 0);
            if (stop || (d > 0 && t >= d)) break;
        }
        hb_finalize_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>((uint32_t)P.n, g->d_comp, sum_d,
                                                                               c_prev, md_dev, ball_dev);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (iterations) *iterations = t;
    return VGA_OK;
}

}  // namespace

// One run with the union launches timed (the autotuner's measurement):
// outputs go to library-owned buffers, *union_ms gets the summed device time
// of the union slices (sparse tables included).
int run_timed(const vga_graph *g, int p, int d, uint64_t seed, const vga_tuning *tune, cudaStream_t stream,
              double *union_ms, int *iterations) {
    DeviceBuffer out;
    VGA_TRY(out.alloc(16 * (size_t)(g->n ? g->n : 1)));
    double *md = out.as<double>();
    return run_impl(g, p, d, seed, 0, md, md + g->n, iterations, nullptr, 0, stream, tune, nullptr, nullptr, -1,
                    union_ms);
}

namespace {

// ---------------------------------------------------------------------------
// Fixed scratch for callers that must not allocate device memory
// (hyperball_run_noalloc).  The array lives in the library's device image:
// every GPU the library is used on holds these bytes from module load until the
// process exits.  Host code must not use its name as a pointer: on the host it
// is only a stand-in for the device symbol, and the device address is looked up
// with cudaGetSymbolAddress once per device context.
// ---------------------------------------------------------------------------
constexpr uint64_t kStaticScratchBytes = 64ull << 20;  // 64 MiB
__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
// Per device: the context the address was looked up in (by its unique ID, which
// a context created later never reuses) and the address.  A device reset or a
// released and re-created primary context loads the module again, possibly at
// another address, so a cached address is used only in the context it came from.
struct StaticScratchSlot {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
StaticScratchSlot g_static_slot[kMaxDevices];

// ID of the context current on this thread, through driver entry points that
// the runtime hands out (no link against the driver library needed).
int current_context_id(unsigned long long *id) {
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q{};
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) {
        set_error("hyperball_run_noalloc: cannot identify the current CUDA context");
        return VGA_ECUDA;
    }
    return VGA_OK;
}

// Device address of g_static_scratch on the current device (`dev`), looked up
// on the first call made in each of that device's contexts.
int static_scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("hyperball_run_noalloc: device %d is beyond the supported %d devices", dev, kMaxDevices);
        return VGA_EINVAL;
    }
    // binds the device's primary context to this thread (created if needed), so
    // that the context queried below is the one the kernels will run in
    VGA_CHECK_CUDA(cudaSetDevice(dev));
    unsigned long long id = 0;
    VGA_TRY(current_context_id(&id));
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticScratchSlot &slot = g_static_slot[dev];
    if (!slot.addr || slot.ctx_id != id) {
        void *addr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
        if (e != cudaSuccess || !addr) {
            set_error("hyperball_run_noalloc: cudaGetSymbolAddress of the fixed scratch failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return VGA_ECUDA;
        }
        slot.addr = addr;
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return VGA_OK;
}

}  // namespace

void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace vga

// Register-range shard (vga_shard_*): slices [s0, s1) of every node's
// counter, with its own union buffers and a full copy of the per-node
// estimator state (identical on every shard).
struct vga_shard {
    const vga_graph *g = nullptr;
    vga::Plan P;  // the graph's plan, with `slices` cut down to this shard's count
    int p = 10;
    uint64_t seed = 0;
    int shard = 0, n_shards = 1;
    uint32_t s0 = 0, s1 = 0, all_slices = 0;
    uint64_t block_bytes = 0, zeros_off = 0;
    vga::DeviceBuffer ws;
    uint8_t *cur = nullptr, *nxt = nullptr, *tab = nullptr;
    double *c_prev = nullptr, *c_cur = nullptr, *sum_d = nullptr, *lc = nullptr;
    uint32_t *flags = nullptr;
    uint8_t *chg = nullptr;                  // change tracking (P.track): change bytes of the shard's slices,
    uint32_t *need = nullptr, *ortab = nullptr;  // need masks and the range-OR table (or per-node masks)
    uint64_t changed_prev = ~0ull;           // (node, slice) pairs the previous pass changed here
    int t = -1;  // passes run; -1 before vga_shard_start
};

using namespace vga;

extern "C" {

int vga_shard_create(const vga_graph *g, int p, uint64_t seed, int shard, int n_shards, const vga_tuning *tuning,
                     vga_shard **out) {
    clear_error();
    if (!g || !out || n_shards < 2 || shard < 0 || shard >= n_shards) {
        set_error("vga_shard_create: need a graph, an output pointer, n_shards >= 2 and 0 <= shard < n_shards");
        return VGA_EINVAL;
    }
    *out = nullptr;
    Plan P;
    VGA_TRY(make_plan(g, p, tuning, &P));
    if (n_shards > P.slices) {
        set_error("vga_shard_create: %d shards but only %d register slices of %d bytes (lower slice_bytes)",
                  n_shards, P.slices, P.S);
        return VGA_EINVAL;
    }
    vga_shard *s = new vga_shard;
    s->g = g;
    s->p = p;
    s->seed = seed;
    s->shard = shard;
    s->n_shards = n_shards;
    s->all_slices = (uint32_t)P.slices;
    s->s0 = (uint32_t)((uint64_t)shard * P.slices / n_shards);
    s->s1 = (uint32_t)((uint64_t)(shard + 1) * P.slices / n_shards);
    P.slices = (int)(s->s1 - s->s0);
    const uint64_t n = P.n, regs = n * P.S * (uint64_t)P.slices;
    uint64_t o = 0;
    const uint64_t off_cur = o;   o = align256(o + regs);
    const uint64_t off_next = o;  o = align256(o + regs);
    const uint64_t off_c0 = o;    o = align256(o + 8 * n);
    const uint64_t off_c1 = o;    o = align256(o + 8 * n);
    const uint64_t off_sum = o;   o = align256(o + 8 * n);
    const uint64_t off_lc = o;    o = align256(o + 8 * ((uint64_t)P.m + 1));
    const uint64_t off_flags = o; o = align256(o + 64);
    const uint64_t off_tab = o;  // the table region, or (mode 1) the keys of pass 1's scatter
    if (P.mode == kModeRuns) o = align256(o + (uint64_t)table_rows(P.scheme) * n * (uint64_t)P.S);
    else if (P.first_scatter) o = align256(o + 4 * n);
    // change tracking over the shard's own slices (a slice's registers depend
    // only on the same slice of the neighbours, so no exchange is needed)
    uint64_t off_chg = 0, off_need = 0, off_ortab = 0;
    if (P.track) {
        P.chg_bytes = align256((uint64_t)P.slices * n);
        off_chg = o;   o = align256(o + P.chg_bytes);
        off_need = o;  o = align256(o + 4 * n);
        off_ortab = o; o = align256(o + 4ull * (P.mode == kModeRuns ? table_rows(P.scheme) : 1) * n);
    }
    const int rc = s->ws.alloc(o);
    if (rc != VGA_OK) {
        delete s;
        return rc;
    }
    uint8_t *base = s->ws.as<uint8_t>();
    s->cur = base + off_cur;
    s->nxt = base + off_next;
    s->c_prev = reinterpret_cast<double *>(base + off_c0);
    s->c_cur = reinterpret_cast<double *>(base + off_c1);
    s->sum_d = reinterpret_cast<double *>(base + off_sum);
    s->lc = reinterpret_cast<double *>(base + off_lc);
    s->flags = reinterpret_cast<uint32_t *>(base + off_flags);
    s->tab = base + off_tab;
    if (P.track) {
        s->chg = base + off_chg;
        s->need = reinterpret_cast<uint32_t *>(base + off_need);
        s->ortab = reinterpret_cast<uint32_t *>(base + off_ortab);
    }
    s->zeros_off = align256(8 * n);
    s->block_bytes = s->zeros_off + align256(4 * n);
    if (P.mode == kModeRuns && n > 0) {
        int r = ensure_run_lookups(g, P.scheme, 0);
        if (r == VGA_OK) {
            P.hub = hub_threshold(g, P.scheme, P.hub_req);
            r = ensure_run_items(g, P.scheme, P.hub, 0, &P.items);
        }
        if (r == VGA_OK && P.group) r = ensure_group_list(g, P.scheme, P.hub, P.group, 0, &P.groups);
        if (r != VGA_OK) {
            delete s;
            return r;
        }
    }
    s->P = P;
    *out = s;
    return VGA_OK;
}

int vga_shard_info(const vga_shard *s, int *slice_first, int *slice_count, int *slice_bytes,
                   uint64_t *partial_bytes) {
    clear_error();
    if (!s) {
        set_error("vga_shard_info: null shard");
        return VGA_EINVAL;
    }
    if (slice_first) *slice_first = (int)s->s0;
    if (slice_count) *slice_count = (int)(s->s1 - s->s0);
    if (slice_bytes) *slice_bytes = s->P.S;
    if (partial_bytes) *partial_bytes = s->block_bytes;
    return VGA_OK;
}

static int shard_partials(vga_shard *s, const uint8_t *regs, void *partial_dev, cudaStream_t stream) {
    const Plan &P = s->P;
    if (!partial_dev || (reinterpret_cast<uintptr_t>(partial_dev) & 255u)) {
        set_error("vga_shard: partial block must be a 256-byte aligned device buffer of vga_shard_info bytes");
        return VGA_EINVAL;
    }
    if (P.n == 0) return VGA_OK;
    uint8_t *blk = static_cast<uint8_t *>(partial_dev);
    const unsigned blocks = (unsigned)((P.n + 7) / 8);
    hb_shard_partial_kernel<<<blocks, 256, 0, stream>>>(regs, (uint32_t)P.n, s->p, P.S, 0u,
                                                        (uint32_t)P.S * (uint32_t)P.slices, P.nib,
                                                        reinterpret_cast<uint64_t *>(blk),
                                                        reinterpret_cast<uint32_t *>(blk + s->zeros_off), s->flags);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

int vga_shard_start(vga_shard *s, void *partial_dev, void *stream_ptr) {
    clear_error();
    if (!s) {
        set_error("vga_shard_start: null shard");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const Plan &P = s->P;
    const uint64_t regs = P.n * P.S * (uint64_t)P.slices;
    const std::vector<double> &table = lc_table(s->p);
    VGA_CHECK_CUDA(cudaMemcpyAsync(s->lc, table.data(), 8 * table.size(), cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(s->flags, 0, 64, stream));
    if (P.n > 0) {
        VGA_CHECK_CUDA(cudaMemsetAsync(s->cur, 0, regs, stream));
        if (P.items.hubs) VGA_CHECK_CUDA(cudaMemsetAsync(s->nxt, 0, regs, stream));
        VGA_CHECK_CUDA(cudaMemsetAsync(s->sum_d, 0, 8 * P.n, stream));
        hb_init_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(
            s->cur, (uint32_t)P.n, s->p, P.S, s->seed, P.nib, s->s0, s->s1,
            P.first_scatter ? static_cast<void *>(s->tab) : nullptr);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_TRY(shard_partials(s, s->cur, partial_dev, stream));
    s->t = 0;
    s->changed_prev = ~0ull;
    return VGA_OK;
}

int vga_shard_union(vga_shard *s, void *partial_dev, uint32_t *changed, void *stream_ptr) {
    clear_error();
    if (!s || s->t < 0) {
        set_error("vga_shard_union: null shard, or vga_shard_start not called");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const Plan &P = s->P;
    uint32_t h[3] = {0, 0, 0};
    bool profiling;
    {
        std::lock_guard<std::mutex> lock(prof().mu);
        profiling = prof().enabled;
    }
    std::vector<PendingTiming> timings;
    struct Settle {
        std::vector<PendingTiming> &t;
        ~Settle() { settle_timings(t, true, nullptr); }
    } settle{timings};
    if (P.n > 0) {
        VGA_CHECK_CUDA(cudaMemsetAsync(s->flags, 0, 4, stream));
        const bool tracked = s->chg && s->t >= 1 &&
                             (P.track == 2 || (double)s->changed_prev < kTrackBelow * (double)P.n * P.slices);
        if (tracked) VGA_TRY(launch_need(P, s->g, s->chg, s->ortab, s->need, stream, profiling ? &timings : nullptr));
        if (s->chg) {
            VGA_CHECK_CUDA(cudaMemsetAsync(s->chg, 0, P.chg_bytes, stream));
            VGA_CHECK_CUDA(cudaMemsetAsync(s->flags + 4, 0, 8, stream));
        }
        if (s->t == 0 && P.first_scatter)
            VGA_TRY(launch_first_pass(P, s->g, s->tab, s->nxt, s->s0, s->s1, s->flags, stream,
                                      profiling ? &timings : nullptr, s->chg));
        else
            VGA_TRY(launch_union(P, s->g, s->cur, s->nxt, s->tab, s->flags, stream, profiling ? &timings : nullptr,
                                 tracked ? s->need : nullptr, s->chg));
        if (s->chg) VGA_TRY(launch_count(P, s->chg, s->flags, stream));
    }
    VGA_TRY(shard_partials(s, s->nxt, partial_dev, stream));
    uint64_t n_changed = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(h, s->flags, 12, cudaMemcpyDeviceToHost, stream));
    if (s->chg) VGA_CHECK_CUDA(cudaMemcpyAsync(&n_changed, s->flags + 4, 8, cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    s->changed_prev = n_changed;
    if (h[2] & 1u) {
        set_error("vga_shard_union: a bounded wait for a TMA copy ran out in pass %d", s->t + 1);
        return VGA_ETIMEOUT;
    }
    if (h[2] & 2u) {
        set_error("vga_shard_union: a partial harmonic sum overflowed 64 bits");
        return VGA_ECORRUPT;
    }
    std::swap(s->cur, s->nxt);
    s->t++;
    if (changed) *changed = h[0] ? 1u : 0u;
    return VGA_OK;
}

int vga_shard_estimate(vga_shard *s, const void *all_partials_dev, uint32_t *increase_flag, void *stream_ptr) {
    clear_error();
    if (!s || s->t < 0 || !all_partials_dev) {
        set_error("vga_shard_estimate: null shard or partials, or vga_shard_start not called");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const Plan &P = s->P;
    uint32_t inc = 0;
    if (P.n > 0) {
        VGA_CHECK_CUDA(cudaMemsetAsync(s->flags + 1, 0, 4, stream));
        const double alpha_mm = hll_alpha_host(s->p) * (double)P.m * (double)P.m;
        double *out = s->t == 0 ? s->c_prev : s->c_cur;  // c_0 is written where c_{t-1} is read next
        hb_shard_estimate_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(
            static_cast<const uint8_t *>(all_partials_dev), s->n_shards, s->block_bytes, s->zeros_off,
            (uint32_t)P.n, s->p, s->t, alpha_mm, s->lc, s->c_prev, out, s->sum_d, s->flags);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        VGA_CHECK_CUDA(cudaMemcpyAsync(&inc, s->flags + 1, 4, cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        if (s->t > 0) std::swap(s->c_prev, s->c_cur);
    }
    if (increase_flag) *increase_flag = inc ? 1u : 0u;
    return VGA_OK;
}

int vga_shard_finalize(vga_shard *s, double *mean_depth_dev, double *ball_size_dev, void *stream_ptr) {
    clear_error();
    if (!s || s->t < 0) {
        set_error("vga_shard_finalize: null shard, or vga_shard_start not called");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const Plan &P = s->P;
    if (P.n > 0) {
        hb_finalize_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(
            (uint32_t)P.n, s->g->d_comp, s->sum_d, s->c_prev, mean_depth_dev, ball_size_dev);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    return VGA_OK;
}

void vga_shard_free(vga_shard *s) { delete s; }

int vga_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(prof().mu);
    prof().enabled = on != 0;
    return VGA_OK;
}

int vga_profile_reset(void) {
    std::lock_guard<std::mutex> lock(prof().mu);
    prof().acc = vga_profile{};
    g_kernel_launches.store(0);
    return VGA_OK;
}

int vga_profile_read(vga_profile *out) {
    clear_error();
    if (!out) {
        set_error("vga_profile_read: null argument");
        return VGA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(prof().mu);
    *out = prof().acc;
    out->kernel_launches = g_kernel_launches.load();
    return VGA_OK;
}

// vga_bench_gather consumer 2: the coalesced L2 stream (stream_bench_kernel)
// over resident_bytes, repeated until about `bytes` have been read; full
// occupancy (4 CTAs of 512 threads per SM).
static int bench_stream(uint64_t resident_bytes, uint64_t bytes, cudaStream_t stream, double *gb_per_s) {
    const uint64_t words = resident_bytes / 16;
    if (words == 0) {
        set_error("vga_bench_gather: buffer below 16 bytes");
        return VGA_EINVAL;
    }
    int dev = 0, sms = 0;
    VGA_CHECK_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t blocks = (uint32_t)std::max(1, sms) * 4, threads = 512;
    const uint32_t passes = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(1u << 20, bytes / (words * 16)));
    DeviceBuffer buf, out;
    VGA_TRY(buf.alloc(words * 16));
    VGA_TRY(out.alloc((uint64_t)blocks * threads / 32 * 4));
    VGA_CHECK_CUDA(cudaMemsetAsync(buf.ptr, 0x5A, words * 16, stream));
    cudaEvent_t e0, e1;
    VGA_CHECK_CUDA(cudaEventCreate(&e0));
    VGA_CHECK_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {  // warm-up (also brings the buffer into L2), then the timed launch
        VGA_CHECK_CUDA(cudaEventRecord(e0, stream));
        stream_bench_kernel<<<blocks, threads, 0, stream>>>(buf.as<uint4>(), words, passes, out.as<uint32_t>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        VGA_CHECK_CUDA(cudaEventRecord(e1, stream));
        VGA_CHECK_CUDA(cudaEventSynchronize(e1));
        VGA_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gb_per_s = (double)words * 16.0 * (double)passes / ((double)ms * 1e-3) / 1e9;
    return VGA_OK;
}

int vga_bench_gather(uint64_t resident_bytes, int chunk_bytes, uint64_t gathers, int consumer, void *stream_ptr,
                     double *gb_per_s) {
    clear_error();
    const int S = chunk_bytes;
    if (!gb_per_s || S < 16 || S > 1024 || (S & (S - 1)) || resident_bytes < (uint64_t)S ||
        resident_bytes / (uint64_t)S > 0xFFFFFFFFull || gathers == 0 || consumer < 0 || consumer > 2) {
        set_error("vga_bench_gather: bad arguments");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    if (consumer == 2) return bench_stream(resident_bytes, (uint64_t)S * gathers, stream, gb_per_s);
    const uint32_t rows = (uint32_t)(resident_bytes / (uint64_t)S);
    const int warps = 8;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const uint32_t blocks = (uint32_t)std::max(1, sms) * 16;
    const uint64_t total_warps = (uint64_t)blocks * warps;
    const uint64_t windows = std::max<uint64_t>(1, gathers / (total_warps * 32));
    DeviceBuffer buf, out;
    VGA_TRY(buf.alloc((uint64_t)rows * S));
    VGA_TRY(out.alloc(total_warps * 4));
    VGA_CHECK_CUDA(cudaMemsetAsync(buf.ptr, 0x5A, (uint64_t)rows * S, stream));
    cudaEvent_t e0, e1;
    VGA_CHECK_CUDA(cudaEventCreate(&e0));
    VGA_CHECK_CUDA(cudaEventCreate(&e1));
    const size_t smem = (size_t)warps * 32 * 4;
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {  // warm-up, then the timed launch
        VGA_CHECK_CUDA(cudaEventRecord(e0, stream));
        switch (S) {
#define VGA_CASE(SS)                                                                                          \
    case SS:                                                                                                  \
        if (consumer)                                                                                         \
            gather_bench_kernel<SS, true><<<blocks, warps * 32, smem, stream>>>(buf.as<uint8_t>(), rows,       \
                                                                                (uint32_t)windows,            \
                                                                                out.as<uint32_t>());          \
        else                                                                                                  \
            gather_bench_kernel<SS, false><<<blocks, warps * 32, smem, stream>>>(buf.as<uint8_t>(), rows,      \
                                                                                 (uint32_t)windows,           \
                                                                                 out.as<uint32_t>());         \
        break;
            VGA_CASE(16)
            VGA_CASE(32)
            VGA_CASE(64)
            VGA_CASE(128)
            VGA_CASE(256)
            VGA_CASE(512)
            VGA_CASE(1024)
#undef VGA_CASE
        }
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        VGA_CHECK_CUDA(cudaEventRecord(e1, stream));
        VGA_CHECK_CUDA(cudaEventSynchronize(e1));
        VGA_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gb_per_s = (double)(total_warps * windows * 32) * (double)S / ((double)ms * 1e-3) / 1e9;
    return VGA_OK;
}

int hyperball_run_noalloc(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth_dev,
                          double *ball_size_dev, int *iterations, void *stream) {
    clear_error();
    if (!g) {
        set_error("hyperball_run_noalloc: null graph");
        return VGA_EINVAL;
    }
    if (p < 4 || p > 16) {
        set_error("hyperball_run_noalloc: precision p = %d is outside 4..16", p);
        return VGA_EINVAL;
    }
    int dev = -1;
    VGA_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) {
        set_error("hyperball_run_noalloc: the graph lives on device %d but device %d is current", g->device, dev);
        return VGA_EINVAL;
    }
    // The per-neighbour union (the run-aware one would allocate its lookup
    // list) at one fixed slice width, so that the scratch size depends on N and
    // p alone, as the header states it, and not on an installed tuning table.
    vga_tuning per_edge{};
    per_edge.union_mode = kModePerEdge;
    per_edge.slice_bytes = (int)std::min<uint32_t>(1u << p, 1024u);
    Plan P;
    VGA_TRY(make_plan(g, p, &per_edge, &P));
    if (P.total > kStaticScratchBytes) {
        set_error("hyperball_run_noalloc: N = %u at p = %d needs %llu bytes of scratch but the fixed scratch holds "
                  "%llu bytes (64 MiB); pass a workspace to hyperball_run_dev instead",
                  g->n, p, (unsigned long long)P.total, (unsigned long long)kStaticScratchBytes);
        return VGA_EINVAL;
    }
    void *scratch = nullptr;
    VGA_TRY(static_scratch_address(dev, &scratch));
    // run_impl zeroes the registers, sum_d and the flags itself and overwrites
    // everything else before reading it, so stale contents of the shared scratch
    // from an earlier call cannot leak into this one.
    const int rc = run_impl(g, p, d, seed, conv_mode, mean_depth_dev, ball_size_dev, iterations, scratch,
                            kStaticScratchBytes, static_cast<cudaStream_t>(stream), &per_edge, nullptr, nullptr, -1);
    // A failure part-way leaves kernels queued that still write the shared
    // array: wait for them, so that a caller who orders calls on the host
    // cannot start the next one while they run.
    if (rc != VGA_OK) cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    return rc;
}

int hyperball_workspace_bytes(const vga_graph *g, int p, uint64_t *bytes) {
    clear_error();
    if (!g || !bytes) {
        set_error("hyperball_workspace_bytes: null argument");
        return VGA_EINVAL;
    }
    Plan P;
    VGA_TRY(make_plan(g, p, nullptr, &P));
    *bytes = P.total;
    return VGA_OK;
}

int hyperball_run_dev(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth_dev,
                      double *ball_size_dev, int *iterations, void *workspace_dev, uint64_t workspace_bytes,
                      void *stream, const vga_tuning *tuning) {
    clear_error();
    return run_impl(g, p, d, seed, conv_mode, mean_depth_dev, ball_size_dev, iterations, workspace_dev,
                    workspace_bytes, static_cast<cudaStream_t>(stream), tuning, nullptr, nullptr, -1);
}

static int run_host_outputs(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth,
                            double *ball_size, int *iterations, uint8_t *trace_regs, double *trace_c, int max_trace,
                            const vga_tuning *tuning) {
    clear_error();
    if (!g) {
        set_error("null graph");
        return VGA_EINVAL;
    }
    DeviceBuffer out;
    VGA_TRY(out.alloc(16 * (size_t)(g->n ? g->n : 1)));
    double *md = out.as<double>();
    double *ball = md + g->n;
    cudaStream_t stream = 0;
    VGA_TRY(run_impl(g, p, d, seed, conv_mode, md, ball, iterations, nullptr, 0, stream, tuning, trace_regs, trace_c,
                     max_trace));
    if (g->n) {
        if (mean_depth) VGA_CHECK_CUDA(cudaMemcpy(mean_depth, md, 8 * (size_t)g->n, cudaMemcpyDeviceToHost));
        if (ball_size) VGA_CHECK_CUDA(cudaMemcpy(ball_size, ball, 8 * (size_t)g->n, cudaMemcpyDeviceToHost));
    }
    return VGA_OK;
}

int hyperball_run(const vga_graph *g, int p, int d, uint64_t seed, double *mean_depth, double *ball_size,
                  int *iterations) {
    return run_host_outputs(g, p, d, seed, 0, mean_depth, ball_size, iterations, nullptr, nullptr, -1, nullptr);
}

int hyperball_run_trace(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth,
                        double *ball_size, int *iterations, uint8_t *regs_host, double *c_host, int max_trace,
                        const vga_tuning *tuning) {
    return run_host_outputs(g, p, d, seed, conv_mode, mean_depth, ball_size, iterations, regs_host, c_host,
                            max_trace, tuning);
}

}  // extern "C"
