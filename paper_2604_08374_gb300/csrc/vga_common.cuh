// vga_common.cuh -- internal declarations shared by the library's translation
// units: the graph object, error reporting, RAII device buffers, and the warp
// LEB128 decoder used by the validation and union kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "vga_hyperball.h"

// Device-resident compressed CSR (Sec. 3.2, "CompressedCsr": u64 byte offsets,
// u32 degrees, the LEB128 byte stream).  The byte buffer is over-allocated by
// kBytePad zero bytes so vector loads near the end stay inside the allocation.
struct vga_graph {
    int device = 0;
    uint32_t n = 0;
    uint64_t n_bytes = 0;
    uint64_t n_edges = 0;
    uint32_t max_degree = 0;
    uint64_t *d_offsets = nullptr;  // n+1
    uint8_t *d_bytes = nullptr;     // n_bytes + kBytePad
    uint32_t *d_degree = nullptr;   // n
    uint32_t *d_comp = nullptr;     // n, or nullptr: every node in one component of size n
    // Range lookups of the run-aware union, per table scheme (runs.cuh), built
    // on first use: node v's lookups are lk[s].d_lk[lk[s].d_off[v] .. d_off[v+1]).
    // Work lists of the run-aware union, one per hub threshold (ensure_run_items).
    struct RunItemSet {
        uint32_t hub_lookups;
        uint64_t count, hub_items;
        uint32_t hubs;
        void *d_items;
    };
    struct RunLookups {
        uint64_t *d_off = nullptr;    // n+1
        uint32_t *d_lk = nullptr;     // total (+ 4 zero entries)
        uint64_t total = 0;
        std::vector<uint64_t> h_off;  // prefix sums of the counts (empty until counted)
        bool ready = false;           // d_off and d_lk built
        std::vector<RunItemSet> items;
        // Grouped lookup lists (ensure_group_list), one per (hub threshold,
        // group size).
        struct GroupSet {
            uint32_t hub_lookups;
            int nodes;
            uint64_t count, rows_total, rows_used, hub_rows;
            void *d_items, *d_rows, *d_cls;
        };
        std::vector<GroupSet> groups;
    };
    mutable std::mutex lk_mu;
    mutable RunLookups lk[2];
    int lk_scheme = 0;  // the table scheme chosen for this graph (counted at load)
    // Optional geometry (host copy): the grid cell of every node on a W x H
    // grid, set by the visibility builder or vga_graph_set_cells.  With it the
    // grouped union forms its groups from 2 x 2 blocks of cells instead of
    // consecutive ids.  Changing it drops the cached group lists.
    int cells_W = 0, cells_H = 0;
    std::vector<uint32_t> cells;
};

namespace vga {

constexpr uint64_t kBytePad = 256;

// Thread-local last-error message (vga_last_error).
void set_error(const char *fmt, ...);
void clear_error();

// Counts one library kernel launch (vga_profile.kernel_launches).
void count_launch();

// HLL alpha_m and the linear-counting table m ln(m/V), V = 0..m (host, cached
// per p), shared by the single-graph and batched paths.
double hll_alpha_host(int p);
const std::vector<double> &lc_table(int p);

#define VGA_CHECK_CUDA(call)                                                                   \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ::vga::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                        \
            return (e_ == cudaErrorMemoryAllocation) ? VGA_ENOMEM : VGA_ECUDA;                 \
        }                                                                                      \
    } while (0)

#define VGA_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != VGA_OK) return rc_; \
    } while (0)

// Owning device allocation, freed on scope exit unless released.
struct DeviceBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer &) = delete;
    DeviceBuffer &operator=(const DeviceBuffer &) = delete;
    ~DeviceBuffer() { reset(); }
    int alloc(size_t nbytes) {
        reset();
        if (nbytes == 0) nbytes = 256;
        cudaError_t e = cudaMalloc(&ptr, nbytes);
        if (e != cudaSuccess) {
            ptr = nullptr;
            set_error("cudaMalloc(%zu bytes) failed: %s", nbytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? VGA_ENOMEM : VGA_ECUDA;
        }
        bytes = nbytes;
        return VGA_OK;
    }
    void reset() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    void *release() {
        void *p = ptr;
        ptr = nullptr;
        bytes = 0;
        return p;
    }
    template <class T>
    T *as() const { return static_cast<T *>(ptr); }
};

// Pinned host scratch for small device->host reads.
struct PinnedBuffer {
    void *ptr = nullptr;
    PinnedBuffer() = default;
    PinnedBuffer(const PinnedBuffer &) = delete;
    ~PinnedBuffer() {
        if (ptr) cudaFreeHost(ptr);
    }
    int alloc(size_t nbytes) {
        cudaError_t e = cudaMallocHost(&ptr, nbytes);
        if (e != cudaSuccess) {
            ptr = nullptr;
            set_error("cudaMallocHost failed: %s", cudaGetErrorString(e));
            return VGA_ENOMEM;
        }
        return VGA_OK;
    }
    template <class T>
    T *as() const { return static_cast<T *>(ptr); }
};

// Range lookups of the run-aware union.  A neighbour list in raster order is a
// sequence of runs of consecutive ids; the maximum over a run [a, a+L) is read
// from a slice's table region: rows T_k[i] = max(cur[i .. i + 2^k)) for the
// window widths 2^k of the graph's table scheme, one N-row level after
// another.  A lookup is the row index r = slot * N + i of T_k[i], slot being
// the level's place in the region.
//   scheme 0: k = 0, 1, 2, 3, 4 (5 rows per node); fewest lookups.
//   scheme 1: k = 0, 2, 4 (3 rows per node); for graphs whose 5-row region
//             would not fit the L2 at 128-byte slices.
constexpr int kRunLevels = 4;  // widest window 2^4 = 16 rows
constexpr int kTableSchemes = 2;
__host__ __device__ constexpr int table_rows(int scheme) { return scheme == 0 ? 5 : 3; }
constexpr int kMaxTableRows = 5;
// r < 5 N must fit in 32 bits.
constexpr uint64_t kRunMaxNodes = 1ull << 29;

// The table scheme for a graph of n nodes on `device`: 1 when a 5-row region
// of 128-byte slices would exceed the grouped union's budget, else 0.
int table_scheme_auto(uint32_t n, int device);
// L2 share the per-node run-aware union's table region aims at (bytes): 3/4
// of the L2.
uint64_t union_l2_budget(int device);
// The same for the grouped union: 5/4 of the L2.  A group reads the rows its
// nodes share together and groups go in block order, so the rows in use at a
// time are a fraction of the region; on the city graph a 151 MB 5-row region
// of 128-byte rows (1.2x the L2) ran faster than the 91 MB 3-row one, while a
// 182 MB region of 256-byte rows or 64-byte rows that fit were slower.
uint64_t grouped_l2_budget(int device);

// One warp's work in the run-aware union: the lookups lk[b .. b + cnt) of node
// v & ~kHubChunk.  A node with more lookups than the hub threshold is split
// into several items flagged kHubChunk, each folding part of the node's
// lookups; they merge into next[v] with a word-wise atomic max.
struct RunItem {
    uint32_t v;
    uint32_t cnt;
    uint64_t b;
};
constexpr uint32_t kHubChunk = 1u << 31;

// Work list of the run-aware union for hub threshold `hub_lookups` (> 0),
// built on first use and held by the graph: the hub chunks first (so that the
// longest work starts first), then every other node in id order.
struct RunItemList {
    const RunItem *items = nullptr;
    uint64_t count = 0, hub_items = 0;
    uint32_t hubs = 0;
};
int ensure_run_items(const vga_graph *g, int scheme, uint32_t hub_lookups, cudaStream_t stream, RunItemList *out);

// Grouped lookup lists of the run-aware union.  The non-hub nodes, in id
// order, are cut into groups of up to kGroupMaxNodes consecutive ones;
// adjacent cells see nearly the same runs, so their lookup lists share many
// entries (about 40 % of a four-node group's at the city size).  Each group's
// lists are merged once per graph into its distinct rows, each tagged with
// its class -- the set of the group's nodes whose list holds it -- and sorted
// by class.  The union then gathers every distinct row once and folds each
// class into one accumulator, merged into the partial maxima of the class's
// nodes when the class ends: the same registers, bit for bit (a max over a
// union of sets), from fewer gathers and fewer folds.
constexpr int kGroupMaxNodes = 8;
struct GroupItem {
    uint32_t node[kGroupMaxNodes];  // the group's nodes (0xffffffff past its end)
    uint64_t b;                     // first row entry in rows[] (a multiple of 4)
    uint32_t cnt;                   // row entries (< 2^31)
    uint32_t nc;                    // classes
    uint64_t cls;                   // first class in cls[] (uint2 {node mask, rows}, in row order)
    uint64_t pad;
};
struct GroupList {
    const GroupItem *items = nullptr;
    uint64_t count = 0;
    const uint32_t *rows = nullptr;  // row indices as in the lookup list (+ 4 zero entries)
    const uint2 *cls = nullptr;
    uint64_t rows_used = 0;          // row entries over all groups (without the padding)
    uint64_t hub_rows = 0;           // lookups of the split hubs, which stay per node
    int nodes = 0;                   // group size
};
int ensure_group_list(const vga_graph *g, int scheme, uint32_t hub_lookups, int nodes, cudaStream_t stream,
                      GroupList *out);

// Automatic hub threshold (lookups per work item): half of one warp's even
// share of a slice's lookups when every SM holds 64 warps, and at least 2048,
// so only nodes that would outlast the rest of a launch are split.  The
// scheme's lookups must have been counted (ensure_run_lookups).
uint32_t hub_lookups_auto(const vga_graph *g, int scheme);

// The first pass's scatter (first_pass_item) keeps one u32 cell per register
// for each of its kFirstPassWarps warps in shared memory: up to
// 4 x (2^13 + 32) x 4 bytes per CTA.
constexpr int kFirstPassMaxP = 13;
constexpr int kFirstPassWarps = 4;

// Autotuner table (autotune.cu): the installed entry for g's degree bucket.
bool tune_table_lookup(const vga_graph *g, vga_tune_entry *out);

// One run with the union launches timed (hyperball.cu), for the autotuner.
int run_timed(const vga_graph *g, int p, int d, uint64_t seed, const vga_tuning *tune, cudaStream_t stream,
              double *union_ms, int *iterations);

// Build the graph's lookup list for a table scheme on first use (thread-safe);
// no-op afterwards.
int ensure_run_lookups(const vga_graph *g, int scheme, cudaStream_t stream);

// Creates a graph object around device offsets and bytes: validates the
// stream on the device, derives degrees, E and the run-aware union's lookup
// counts.  Takes ownership of the device pointers on success (and frees them
// on failure).  With h_bytes (and h_offsets) given, d_bytes is still empty
// apart from its zeroed padding, and the bytes are copied from the host here,
// in chunks overlapped with the validation of the nodes already complete.
int finish_graph_load(uint32_t n, uint64_t n_bytes, uint64_t *d_offsets, uint8_t *d_bytes, const uint32_t *comp_host,
                      cudaStream_t stream, vga_graph **out, const uint64_t *h_offsets = nullptr,
                      const uint8_t *h_bytes = nullptr);

// ---------------------------------------------------------------------------
// Warp LEB128 window decoder (Sec. 3.2 encoding; the paper decodes each list
// with one thread into shared memory, here a whole warp decodes 32 bytes per
// step).  The window starts on a varint boundary at `pos`; lane i holds byte
// pos+i.  Terminators (high bit clear) are found with a ballot, each
// terminator lane assembles its varint from up to four preceding bytes with
// shuffles, and an inclusive warp scan of the values turns first-absolute /
// then-delta values into ids.  Varints that do not end inside the window are
// left for the next step.
// ---------------------------------------------------------------------------
template <class Id>
struct WindowDecode {
    uint32_t term_mask;  // lanes holding the last byte of a complete varint
    int advance;         // bytes consumed (last terminator lane + 1), 0 if none
    Id id;               // per lane: decoded id (valid on terminator lanes)
    Id next_base;        // id of the window's last complete varint
    uint32_t value;      // per lane: the varint's value (terminator lanes)
    int bad;             // per lane: varint longer than 5 bytes or above 32 bits
};

// Id = uint32_t for the hot path (graphs are validated at load); uint64_t for
// validation, so that a wrapping sum is seen rather than hidden.
template <class Id>
__device__ __forceinline__ WindowDecode<Id> decode_window(const uint8_t *__restrict__ bytes, uint64_t pos,
                                                          uint64_t end, Id base, int lane) {
    WindowDecode<Id> r;
    const bool in = pos + (uint64_t)lane < end;
    const uint32_t b = in ? (uint32_t)__ldg(bytes + pos + lane) : 0x80u;
    const bool term = in && !(b & 0x80u);
    const uint32_t T = __ballot_sync(0xffffffffu, term);
    r.term_mask = T;
    r.advance = T ? 32 - __clz(T) : 0;
    const uint32_t b1 = __shfl_up_sync(0xffffffffu, b, 1);
    const uint32_t b2 = __shfl_up_sync(0xffffffffu, b, 2);
    const uint32_t b3 = __shfl_up_sync(0xffffffffu, b, 3);
    const uint32_t b4 = __shfl_up_sync(0xffffffffu, b, 4);
    const uint32_t below = T & ((1u << lane) - 1u);
    const int start = below ? 32 - __clz(below) : 0;
    const int len = lane - start + 1;
    uint64_t v = 0;
    r.bad = 0;
    if (term) {
        v = b & 0x7Fu;
        if (len >= 2) v = (v << 7) | (b1 & 0x7Fu);
        if (len >= 3) v = (v << 7) | (b2 & 0x7Fu);
        if (len >= 4) v = (v << 7) | (b3 & 0x7Fu);
        if (len >= 5) v = (v << 7) | (b4 & 0x7Fu);
        if (len > 5 || v > 0xFFFFFFFFull) r.bad = 1;
    }
    r.value = (uint32_t)v;
    Id s = (Id)(uint32_t)v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Id t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    r.id = base + s;
    r.next_base = T ? __shfl_sync(0xffffffffu, r.id, r.advance - 1) : base;
    return r;
}


__device__ __forceinline__ uint4 vmax4(uint4 a, uint4 b) {
    return make_uint4(__vmaxu4(a.x, b.x), __vmaxu4(a.y, b.y), __vmaxu4(a.z, b.z), __vmaxu4(a.w, b.w));
}

}  // namespace vga
