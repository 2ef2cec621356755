// visibility.cu -- visibility graph of an obstacle grid, built on the device
// (Sec. 3.1).  Two free cells see each other iff the closed segment between
// their centres meets no obstacle cell's closed square.  Nodes are the cells of
// the largest 4-connected free component, numbered in raster order (Sec. 3.2),
// so neighbour lists come out sorted and delta-encode into mostly one-byte
// LEB128 varints.
//
// Method: the angular sweep of Sec. 3.1 ("SparkSieve angular sweep": per
// source, eight octants expand outwards while a list of open gaps in
// tan-space [0, 1] loses the ranges obstacles cover), with the gaps' ends kept
// as exact integer fractions so that the result equals the pairwise rule above
// for every pair.  Pipeline: (host) main component and numbering, obstacle
// bitmaps; (device) count pass: per source, the octants swept into a node
// bitmap and the LEB128 bytes of its list counted; (host) prefix sum into
// offsets; (device) write pass: the same sweep, the bytes written; then the
// ordinary load path validates the stream and derives degrees.
#include <algorithm>
#include <utility>
#include <vector>

#include "vga_common.cuh"

namespace vga {
namespace {

constexpr int kMaxSide = 16384;

// Largest 4-connected free component (ties: lowest raster index), numbered in
// raster order.  Returns the raster cell of every node.
std::vector<uint32_t> main_component_cells(int W, int H, const uint8_t *obst) {
    const size_t C = (size_t)W * H;
    std::vector<int32_t> label(C, -1);
    std::vector<uint32_t> queue;
    queue.reserve(C);
    int32_t best = -1, next = 0;
    size_t best_size = 0;
    for (size_t c = 0; c < C; c++) {
        if (obst[c] || label[c] >= 0) continue;
        const int32_t L = next++;
        queue.clear();
        queue.push_back((uint32_t)c);
        label[c] = L;
        for (size_t head = 0; head < queue.size(); head++) {
            const uint32_t cur = queue[head];
            const int x = (int)(cur % (uint32_t)W), y = (int)(cur / (uint32_t)W);
            const int nb[4][2] = {{x - 1, y}, {x + 1, y}, {x, y - 1}, {x, y + 1}};
            for (auto &q : nb) {
                if (q[0] < 0 || q[1] < 0 || q[0] >= W || q[1] >= H) continue;
                const size_t nc = (size_t)q[1] * W + q[0];
                if (obst[nc] || label[nc] >= 0) continue;
                label[nc] = L;
                queue.push_back((uint32_t)nc);
            }
        }
        if (queue.size() > best_size) {
            best_size = queue.size();
            best = L;
        }
    }
    std::vector<uint32_t> cells;
    cells.reserve(best_size);
    for (size_t c = 0; c < C; c++)
        if (best >= 0 && label[c] == best) cells.push_back((uint32_t)c);
    return cells;
}

// Hilbert-curve position of (x, y) in a 2^k x 2^k square (Sec. 3.2, optional
// Hilbert reordering): walk the levels from the coarsest; each level adds its
// quadrant's rank in curve order (0, 1, 2, 3 for lower-left, upper-left,
// upper-right, lower-right in the current frame) times the quadrant size, then
// maps the point into that quadrant's own frame (the lower quadrants are
// transposed, the lower-right one also mirrored).
uint64_t hilbert_position(int k, uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (int lvl = k - 1; lvl >= 0; lvl--) {
        const uint32_t half = 1u << lvl;
        const uint32_t qx = (x >> lvl) & 1u, qy = (y >> lvl) & 1u;
        const uint32_t rank = qx ? (qy ? 2u : 3u) : (qy ? 1u : 0u);
        d += (uint64_t)rank << (2 * lvl);
        x &= half - 1u;
        y &= half - 1u;
        if (!qy) {
            if (qx) {
                x = half - 1u - x;
                y = half - 1u - y;
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// ---------------------------------------------------------------------------
// The sweep.  From a source s, each of the 8 octants is swept column by column
// outwards.  In octant coordinates a cell is (k, r): k >= 0 steps along the
// major axis, 0 <= r <= k + 1 along the minor one.  The closed square of an
// obstacle at (k, r) is seen from s's centre under the closed range of slopes
// (minor / major) [(2r - 1) / (2k + 1), (2r + 1) / (2k - 1)] (k >= 1), so the
// slopes in [0, 1] that no obstacle of columns 0 .. k - 1 blocks form a list of
// disjoint intervals, each end open or closed.  A target (k, r) is visible iff
// r / k lies in one of them, except that the target on the diagonal (r = k)
// is also blocked by the obstacle (k, k - 1), which its segment touches at a
// corner inside column k.  After column k's targets, each interval loses the
// slope ranges of the column's obstacles in rows a - 1 .. b + 1 (a .. b being
// the interval's target rows; no other row's range meets it); the remaining
// pieces carry on to column k + 1.  Every blocking range is at least 1/k wide,
// so at most k + 1 intervals are alive at column k + 1.
// ---------------------------------------------------------------------------

constexpr int kSweepWarps = 8;                     // one warp per octant
constexpr int kSweepThreads = kSweepWarps * 32;
constexpr int kSweepCap = 48;                      // intervals per list in shared memory
constexpr int kPad = 64;                           // margin bits (obstacles) on both sides of a line
constexpr uint32_t kNoSource = 0xffffffffu;

// Test hooks: a smaller shared-memory list capacity sends more sources down
// the global-list retry; a node limit moves the node bitmap to global memory.
int g_sweep_smem_cap = kSweepCap;
uint32_t g_sweep_smem_bitmap_nodes = 0;   // 0: as many as shared memory allows

// A slope n / d (d > 0) with its end open or closed.
struct Slope {
    int n, d;
    bool open;
};

__device__ __forceinline__ int slope_cmp(const Slope &a, const Slope &b) {
    const int l = a.n * b.d, r = b.n * a.d;   // |numerators|, denominators < 2^15
    return l < r ? -1 : (l > r ? 1 : 0);
}

__device__ __forceinline__ bool interval_nonempty(const Slope &lo, const Slope &hi) {
    const int c = slope_cmp(lo, hi);
    return c < 0 || (c == 0 && !lo.open && !hi.open);
}

// Stored slopes lie in [0, 1] with denominators below 2^15 (sides <= 16384).
__device__ __forceinline__ uint32_t slope_pack(const Slope &s) {
    return (uint32_t)s.n | ((uint32_t)s.d << 15) | (s.open ? 1u << 30 : 0u);
}
__device__ __forceinline__ Slope slope_unpack(uint32_t w) {
    return Slope{(int)(w & 0x7fffu), (int)((w >> 15) & 0x7fffu), ((w >> 30) & 1u) != 0};
}

struct SweepArgs {
    const uint32_t *rowbits;   // H lines of words_r words: bit x + kPad of line y = obstacle (x, y)
    const uint32_t *colbits;   // W lines of words_c words: bit y + kPad of line x = obstacle (x, y)
    int W, H, words_r, words_c;
    const int32_t *node_of_cell;   // W * H: node id, or -1 off the main component
    const uint32_t *cells;         // n: raster cell of each node
    uint32_t n;
    const uint32_t *sources;       // the sources to sweep (nullptr: nodes 0 .. count - 1)
    uint32_t count;
    uint32_t *next;                // work counter, zero at launch
    uint64_t *row_bytes;           // count pass: bytes of each source's list
    const uint64_t *offsets;       // write pass: each list's first byte
    uint8_t *out;
    uint32_t *retry, *retry_count; // sources whose interval lists outgrew shared memory
    uint2 *glists;                 // global interval lists (cap glist_cap each, 2 per warp)
    int glist_cap;
    uint32_t *gbitmap;             // global node bitmaps, words_n per CTA (large graphs)
    uint32_t words_n;              // ceil(n / 32)
    int mask_words;                // row-mask (and staged obstacle) words per warp
    int smem_cap;                  // interval-list capacity in shared memory (<= kSweepCap)
    int *err;                      // nonzero: a visible cell off the component, or a list overflow
};

// 32 obstacle bits of a line starting at bit pos (pos >= 0, within the margins).
// Positions past a line's ends read as obstacles, like its margins.
__device__ __forceinline__ uint32_t line_bits32(const uint32_t *__restrict__ line, int lw, int pos) {
    if (pos < 0 || (pos >> 5) + 1 >= lw) return 0xffffffffu;
    const int w = pos >> 5, s = pos & 31;
    return __funnelshift_r(__ldg(line + w), __ldg(line + w + 1), s);
}

// Obstacle bits of rows r0 .. r0 + 31 of one octant column (bit j = row r0 + j).
__device__ __forceinline__ uint32_t column_bits(const uint32_t *__restrict__ line, int lw, int c0, bool neg, int r0) {
    return neg ? __brev(line_bits32(line, lw, c0 - r0 - 31)) : line_bits32(line, lw, c0 + r0);
}

__device__ __forceinline__ bool column_obst(const uint32_t *__restrict__ line, int lw, int c0, bool neg, int r) {
    const int pos = neg ? c0 - r : c0 + r;
    if (pos < 0 || (pos >> 5) >= lw) return true;
    return (__ldg(line + (pos >> 5)) >> (pos & 31)) & 1u;
}

// Rows a .. b of column k whose slopes r / k lie in [lo, hi] (b < a: none).
// Numerators are at most 2k + 3 and k < 2^14, so the products fit 32 bits.
__device__ __forceinline__ void interval_rows(const Slope &lo, const Slope &hi, int k, int &a, int &b) {
    const uint32_t nl = (uint32_t)lo.n * (uint32_t)k, nh = (uint32_t)hi.n * (uint32_t)k;
    uint32_t qa = (nl + (uint32_t)lo.d - 1u) / (uint32_t)lo.d;
    if (lo.open && qa * (uint32_t)lo.d == nl) qa++;
    const uint32_t qb = nh / (uint32_t)hi.d;
    a = (int)qa;
    b = (int)qb - ((hi.open && qb * (uint32_t)hi.d == nh) ? 1 : 0);
}

// Obstacle bits of rows y .. y + 31 of the current column from its words
// staged in shared memory (obw[w] holds rows 32w .. 32w + 31).
__device__ __forceinline__ uint32_t staged_bits(const uint32_t *obw, int y) {
    return __funnelshift_r(obw[y >> 5], obw[(y >> 5) + 1], y & 31);
}

// Appends to out (through the warp's counter) the pieces of interval
// [lo, hi] left after the obstacles of column k in rows r0 .. r1 (read from
// the column's staged words); pieces past cap are counted but not stored.
__device__ void interval_pieces(Slope lo, const Slope &hi, int k, int r0, int r1, const uint32_t *obw, uint2 *out,
                                int *count, int cap) {
    int y = r0;
    while (y <= r1) {
        const int lim = min(32, r1 - y + 1);
        const uint32_t valid = lim == 32 ? 0xffffffffu : ((1u << lim) - 1u);
        const uint32_t ob = staged_bits(obw, y) & valid;
        if (!ob) {
            y += lim;
            continue;
        }
        const int s = y + __ffs(ob) - 1;
        // the run's last obstacle row: the row before the next free one
        int e = r1;
        for (int z = s; z <= r1;) {
            const int lim2 = min(32, r1 - z + 1);
            const uint32_t valid2 = lim2 == 32 ? 0xffffffffu : ((1u << lim2) - 1u);
            const uint32_t fr = ~staged_bits(obw, z) & valid2;
            if (fr) {
                e = z + __ffs(fr) - 2;
                break;
            }
            z += lim2;
        }
        const Slope mn{2 * s - 1, 2 * k + 1, true}, mx{2 * e + 1, 2 * k - 1, true};
        const Slope phi = slope_cmp(hi, mn) < 0 ? hi : mn;
        if (interval_nonempty(lo, phi)) {
            const int at = atomicAdd(count, 1);
            if (at < cap) out[at] = make_uint2(slope_pack(lo), slope_pack(phi));
        }
        const int c2 = slope_cmp(mx, lo);
        if (c2 > 0) lo = mx;
        else if (c2 == 0) lo.open = true;
        y = e + 1;
    }
    if (interval_nonempty(lo, hi)) {
        const int at = atomicAdd(count, 1);
        if (at < cap) out[at] = make_uint2(slope_pack(lo), slope_pack(hi));
    }
}

__device__ __forceinline__ uint32_t varint_len(uint32_t x) {
    return x < (1u << 7) ? 1u : x < (1u << 14) ? 2u : x < (1u << 21) ? 3u : x < (1u << 28) ? 4u : 5u;
}

// One warp sweeps octant `oct` of source (sx, sy), setting the bits of the
// visible nodes in bm.  Returns false when the interval list outgrew cap.
__device__ bool sweep_octant(const SweepArgs &A, int oct, int sx, int sy, uint32_t *bm, uint2 *la, uint2 *lb,
                             int cap, uint32_t *mask, uint32_t *obw, int *count, int &id_lo, int &id_hi) {
    const int lane = threadIdx.x & 31;
    const bool xmajor = (oct >> 2) == 0;
    const int smaj = (oct & 1) ? -1 : 1;
    const bool neg = (oct & 2) != 0;
    const int smin = neg ? -1 : 1;
    const int maj0 = xmajor ? sx : sy, min0 = xmajor ? sy : sx;
    const int maj_n = xmajor ? A.W : A.H;
    const uint32_t *base = xmajor ? A.colbits : A.rowbits;
    const int lw = xmajor ? A.words_c : A.words_r;
    const int c0 = min0 + kPad;
    // column 0: the obstacle (0, 1) blocks slope 1 and beyond
    if (lane == 0) {
        const bool o01 = column_obst(base + (size_t)maj0 * lw, lw, c0, neg, 1);
        la[0] = make_uint2(slope_pack(Slope{0, 1, false}), slope_pack(Slope{1, 1, o01}));
    }
    __syncwarp();
    int na = 1;
    for (int k = 1; na > 0; k++) {
        const int maj = maj0 + smaj * k;
        if (maj < 0 || maj >= maj_n) break;
        const uint32_t *line = base + (size_t)maj * lw;
        // 1. the target rows of every interval into the row mask
        int amin = 0x7fffffff, bmax = -1, rmax = 0;
        int a0 = 0, b0 = -1;   // rows of this lane's first interval, kept for step 3
        for (int i = lane; i < na; i += 32) {
            const uint2 iv = la[i];
            const Slope lo = slope_unpack(iv.x), hi = slope_unpack(iv.y);
            int a, b;
            interval_rows(lo, hi, k, a, b);
            if (i == lane) {
                a0 = a;
                b0 = b;
            }
            if (b >= A.mask_words * 32 - 33) {   // b <= k < the major extent: never taken
                atomicOr(A.err, 4);
                b = A.mask_words * 32 - 34;
            }
            rmax = max(rmax, b + 1);
            if (a <= b) {
                amin = min(amin, a);
                bmax = max(bmax, b);
                for (int w = a >> 5; w <= (b >> 5); w++) {
                    const int lo_b = max(a - w * 32, 0), hi_b = min(b - w * 32, 31);
                    const uint32_t bits = (hi_b == 31 ? 0xffffffffu : ((1u << (hi_b + 1)) - 1u)) & ~((1u << lo_b) - 1u);
                    atomicOr(mask + w, bits);
                }
            }
        }
        amin = __reduce_min_sync(0xffffffffu, amin);
        bmax = __reduce_max_sync(0xffffffffu, bmax);
        rmax = __reduce_max_sync(0xffffffffu, rmax);
        // the column's obstacle words for rows 0 .. rmax + 32, staged once for
        // steps 2 and 3
        for (int w = lane; w <= (rmax >> 5) + 1; w += 32) obw[w] = column_bits(line, lw, c0, neg, w * 32);
        __syncwarp();
        // 2. visible targets: masked rows that are free; the diagonal target
        //    also needs (k, k - 1) free
        if (bmax >= 0) {
            const bool diag_blocked = column_obst(line, lw, c0, neg, k - 1);
            for (int w = amin >> 5; w <= (bmax >> 5); w++) {
                const uint32_t m = mask[w];
                uint32_t vis = m & ~obw[w];
                if (diag_blocked && k >= w * 32 && k < w * 32 + 32) vis &= ~(1u << (k - w * 32));
                if ((vis >> lane) & 1u) {
                    const int r = w * 32 + lane;
                    const int x = xmajor ? maj : sx + smin * r;
                    const int y = xmajor ? sy + smin * r : maj;
                    const int id = __ldg(A.node_of_cell + (size_t)y * A.W + x);
                    if (id >= 0) {
                        atomicOr(bm + (id >> 5), 1u << (id & 31));
                        id_lo = min(id_lo, id);
                        id_hi = max(id_hi, id);
                    } else {
                        atomicOr(A.err, 1);
                    }
                }
                __syncwarp();
                if (lane == 0) mask[w] = 0u;
            }
        }
        __syncwarp();
        // 3. the pieces each interval leaves for column k + 1, appended to
        //    the other list in any order
        if (lane == 0) *count = 0;
        __syncwarp();
        for (int i = lane; i < na; i += 32) {
            const uint2 iv = la[i];
            const Slope lo = slope_unpack(iv.x), hi = slope_unpack(iv.y);
            int a = a0, b = b0;
            if (i != lane) interval_rows(lo, hi, k, a, b);
            interval_pieces(lo, hi, k, max(a - 1, 0), b + 1, obw, lb, count, cap);
        }
        __syncwarp();
        const int total = *count;
        if (total > cap) return false;
        uint2 *t = la;
        la = lb;
        lb = t;
        na = total;
    }
    return true;
}

// Persistent CTAs of 8 warps take sources from a counter; each warp sweeps
// one octant into the CTA's node bitmap, then the warps encode the bitmap's
// set bits as the source's LEB128 delta list (WRITE = false: count the bytes
// only).  GLOBAL_LISTS: interval lists in global memory with room for the
// proven maximum (retried sources); otherwise kSweepCap entries in shared
// memory, and a source whose list outgrows them is queued for the retry.
template <bool WRITE, bool GLOBAL_LISTS, bool SMEM_BITMAP>
__global__ void __launch_bounds__(kSweepThreads, 6) visibility_sweep_kernel(SweepArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_src;
    __shared__ int s_overflow, s_lo[kSweepWarps], s_hi[kSweepWarps];
    __shared__ int s_first[kSweepWarps], s_last[kSweepWarps];
    __shared__ uint32_t s_bytes[kSweepWarps];
    __shared__ int s_count[kSweepWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *p = smem;
    uint32_t *bm;
    if (SMEM_BITMAP) {
        bm = reinterpret_cast<uint32_t *>(p);
        p += (size_t)((A.words_n + 3) & ~3u) * 4;
    } else {
        bm = A.gbitmap + (size_t)blockIdx.x * A.words_n;
    }
    uint2 *la, *lb;
    int cap;
    if (GLOBAL_LISTS) {
        la = A.glists + ((size_t)blockIdx.x * kSweepWarps + warp) * 2 * A.glist_cap;
        lb = la + A.glist_cap;
        cap = A.glist_cap;
    } else {
        la = reinterpret_cast<uint2 *>(p) + (size_t)warp * 2 * kSweepCap;
        lb = la + kSweepCap;
        cap = A.smem_cap;
        p += (size_t)kSweepWarps * 2 * kSweepCap * sizeof(uint2);
    }
    uint32_t *mask = reinterpret_cast<uint32_t *>(p) + (size_t)warp * A.mask_words;
    uint32_t *obw = reinterpret_cast<uint32_t *>(p) + (size_t)(kSweepWarps + warp) * A.mask_words;
    for (uint32_t w = threadIdx.x; w < A.words_n; w += blockDim.x) bm[w] = 0u;
    for (int w = lane; w < A.mask_words; w += 32) mask[w] = 0u;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(A.next, 1u);
            s_src = i < A.count ? (A.sources ? A.sources[i] : i) : kNoSource;
            s_overflow = 0;
        }
        __syncthreads();
        const uint32_t u = s_src;
        if (u == kNoSource) break;
        const uint32_t cell = A.cells[u];
        const int sx = (int)(cell % (uint32_t)A.W), sy = (int)(cell / (uint32_t)A.W);
        int id_lo = 0x7fffffff, id_hi = -1;
        if (!sweep_octant(A, warp, sx, sy, bm, la, lb, cap, mask, obw, &s_count[warp], id_lo, id_hi)) {
            if (lane == 0) s_overflow = 1;
            for (int w = lane; w < A.mask_words; w += 32) mask[w] = 0u;
        }
        id_lo = __reduce_min_sync(0xffffffffu, id_lo);
        id_hi = __reduce_max_sync(0xffffffffu, id_hi);
        if (lane == 0) {
            s_lo[warp] = id_lo;
            s_hi[warp] = id_hi;
        }
        __syncthreads();
        int lo = 0x7fffffff, hi = -1;
#pragma unroll
        for (int w = 0; w < kSweepWarps; w++) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        const bool overflow = s_overflow != 0;
        if (hi >= 0 && !overflow) {
            // encode: warp w takes an equal share of the bitmap words lo/32 .. hi/32
            const uint32_t w0 = (uint32_t)lo >> 5, w1 = ((uint32_t)hi >> 5) + 1;
            const uint32_t per = (w1 - w0 + kSweepWarps - 1) / kSweepWarps;
            const uint32_t mb = min(w0 + warp * per, w1), me = min(mb + per, w1);
            // phase A: first and last id of the share, and its bytes without
            // the leading varint of its first id
            int first = -1, last = -1;
            uint32_t bytes = 0;
            for (uint32_t c = mb; c < me; c += 32) {
                const uint32_t wi = c + lane;
                const uint32_t word = wi < me ? (SMEM_BITMAP ? bm[wi] : __ldcg(bm + wi)) : 0u;
                const int wl = word ? (int)(wi * 32 + 31 - __clz(word)) : -1;
                const int wf = word ? (int)(wi * 32 + __ffs(word) - 1) : 0x7fffffff;
                int incl = wl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o && t > incl) incl = t;
                }
                int excl = __shfl_up_sync(0xffffffffu, incl, 1);
                if (lane == 0) excl = -1;
                if (last > excl) excl = last;
                uint32_t nb = 0;
                if (word) {
                    nb = (uint32_t)__popc(word) - 1u;
                    if (excl >= 0) nb += varint_len((uint32_t)(wf - excl));
                }
                bytes += __reduce_add_sync(0xffffffffu, nb);
                const int cf = __reduce_min_sync(0xffffffffu, wf);
                if (first < 0 && cf != 0x7fffffff) first = cf;
                const int cl = __shfl_sync(0xffffffffu, incl, 31);
                if (cl > last) last = cl;
            }
            if (lane == 0) {
                s_first[warp] = first;
                s_last[warp] = last;
                s_bytes[warp] = bytes;
            }
            __syncthreads();
            // each share's leading varint follows the last id of the shares before it
            int prev = -1, run = -1;
            uint64_t start = 0, total = 0;
            for (int w = 0; w < kSweepWarps; w++) {
                if (w == warp) prev = run;
                uint32_t bw = s_bytes[w];
                if (s_first[w] >= 0) bw += varint_len(run < 0 ? (uint32_t)s_first[w] : (uint32_t)(s_first[w] - run));
                if (w < warp) start += bw;
                total += bw;
                if (s_last[w] > run) run = s_last[w];
            }
            if (!WRITE) {
                if (threadIdx.x == 0) A.row_bytes[u] = total;
            } else {
                // phase B: write the share's varints from its first byte on
                uint64_t pos = A.offsets[u] + start;
                const uint64_t end = A.offsets[u + 1];
                int run_prev = prev;
                for (uint32_t c = mb; c < me; c += 32) {
                    const uint32_t wi = c + lane;
                    const uint32_t word = wi < me ? (SMEM_BITMAP ? bm[wi] : __ldcg(bm + wi)) : 0u;
                    const int wl = word ? (int)(wi * 32 + 31 - __clz(word)) : -1;
                    int incl = wl;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o && t > incl) incl = t;
                    }
                    int excl = __shfl_up_sync(0xffffffffu, incl, 1);
                    if (lane == 0) excl = -1;
                    if (run_prev > excl) excl = run_prev;
                    uint32_t nb = 0;
                    if (word) {
                        const uint32_t wf = wi * 32 + (__ffs(word) - 1);
                        nb = (uint32_t)__popc(word) - 1u + varint_len(excl < 0 ? wf : wf - (uint32_t)excl);
                    }
                    uint32_t sc = nb;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(0xffffffffu, sc, o);
                        if (lane >= o) sc += t;
                    }
                    if (word) {
                        uint64_t q = pos + (sc - nb);
                        uint32_t left = word;
                        int last_id = excl;
                        while (left) {
                            const uint32_t id = wi * 32 + (__ffs(left) - 1);
                            left &= left - 1u;
                            uint32_t x = last_id < 0 ? id : id - (uint32_t)last_id;
                            do {
                                uint8_t byte = (uint8_t)(x & 0x7fu);
                                x >>= 7;
                                if (x) byte |= 0x80u;
                                if (q < end) A.out[q] = byte;   // the count pass sized the list
                                else atomicOr(A.err, 8);
                                q++;
                            } while (x);
                            last_id = (int)id;
                        }
                    }
                    pos += __shfl_sync(0xffffffffu, sc, 31);
                    const int cl = __shfl_sync(0xffffffffu, incl, 31);
                    if (cl > run_prev) run_prev = cl;
                }
            }
        } else if (!WRITE && threadIdx.x == 0) {
            A.row_bytes[u] = 0;
        }
        if (overflow && threadIdx.x == 0) {
            if (GLOBAL_LISTS) {
                atomicOr(A.err, 2);
            } else if (!WRITE) {
                A.retry[atomicAdd(A.retry_count, 1u)] = u;
            }
        }
        // every warp has read its share: clear the words this source set (a
        // global bitmap is set by atomics in the L2, so it is read and
        // cleared there, past the L1)
        __syncthreads();
        if (hi >= 0)
            for (uint32_t w = ((uint32_t)lo >> 5) + threadIdx.x; w <= ((uint32_t)hi >> 5); w += blockDim.x) {
                if (SMEM_BITMAP) bm[w] = 0u;
                else __stcg(bm + w, 0u);
            }
        __syncthreads();
    }
}

}  // namespace
}  // namespace vga

using namespace vga;

extern "C" {

int vga_visibility_count(int W, int H, const uint8_t *obst, uint32_t *n_nodes) {
    clear_error();
    if (!obst || !n_nodes || W < 1 || H < 1 || W > kMaxSide || H > kMaxSide) {
        set_error("vga_visibility_count: bad arguments (W=%d, H=%d)", W, H);
        return VGA_EINVAL;
    }
    *n_nodes = (uint32_t)main_component_cells(W, H, obst).size();
    return VGA_OK;
}

int vga_visibility_build_ordered(int W, int H, const uint8_t *obst, int order, uint64_t *cell_of_node,
                                 vga_graph **out) {
    clear_error();
    if (!obst || !out || W < 1 || H < 1 || W > kMaxSide || H > kMaxSide || (order != 0 && order != 1)) {
        set_error("vga_visibility_build: bad arguments (W=%d, H=%d, order=%d, limit %d)", W, H, order, kMaxSide);
        return VGA_EINVAL;
    }
    std::vector<uint32_t> cells = main_component_cells(W, H, obst);
    if (order == 1) {
        int k = 1;
        while ((1 << k) < std::max(W, H)) k++;
        std::vector<std::pair<uint64_t, uint32_t>> keyed(cells.size());
        for (size_t i = 0; i < cells.size(); i++)
            keyed[i] = {hilbert_position(k, cells[i] % (uint32_t)W, cells[i] / (uint32_t)W), cells[i]};
        std::sort(keyed.begin(), keyed.end());
        for (size_t i = 0; i < cells.size(); i++) cells[i] = keyed[i].second;
    }
    const uint32_t n = (uint32_t)cells.size();
    if (cell_of_node)
        for (uint32_t v = 0; v < n; v++) cell_of_node[v] = cells[v];
    // obstacle bitmaps with kPad margin bits of obstacles on both ends of
    // every line: row-major lines for the octants that step along y, and
    // column-major ones for those that step along x
    const int words_r = (W + 2 * kPad + 31) / 32, words_c = (H + 2 * kPad + 31) / 32;
    std::vector<uint32_t> rowbits((size_t)H * words_r, 0xffffffffu), colbits((size_t)W * words_c, 0xffffffffu);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            if (!obst[(size_t)y * W + x]) {
                const int pr = x + kPad, pc = y + kPad;
                rowbits[(size_t)y * words_r + (pr >> 5)] &= ~(1u << (pr & 31));
                colbits[(size_t)x * words_c + (pc >> 5)] &= ~(1u << (pc & 31));
            }
    std::vector<int32_t> node_of_cell((size_t)W * H, -1);
    for (uint32_t v = 0; v < n; v++) node_of_cell[cells[v]] = (int32_t)v;
    const int maxdim = std::max(W, H);
    const uint32_t words_n = (n + 31) / 32;
    const int mask_words = maxdim / 32 + 2;
    int dev = 0, sms = 0, smem_optin = 0;
    VGA_CHECK_CUDA(cudaGetDevice(&dev));
    VGA_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VGA_CHECK_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t list_smem = (size_t)kSweepWarps * 2 * kSweepCap * sizeof(uint2);
    const size_t mask_smem = (size_t)2 * kSweepWarps * mask_words * 4;   // row masks and staged obstacle words
    const size_t bitmap_smem = (size_t)((words_n + 3) & ~3u) * 4;
    // the node bitmap stays in shared memory while two CTAs fit an SM
    const bool smem_bitmap = bitmap_smem + list_smem + mask_smem + 1024 <= (size_t)smem_optin / 2 &&
                             (g_sweep_smem_bitmap_nodes == 0 || n <= g_sweep_smem_bitmap_nodes);
    const int glist_cap = maxdim + 2;   // at most k + 1 intervals are alive at column k + 1

    DeviceBuffer d_rowbits, d_colbits, d_noc, d_cells, d_rowbytes, d_counter, d_retry, d_err, d_gbitmap, d_glists;
    VGA_TRY(d_rowbits.alloc(rowbits.size() * 4));
    VGA_TRY(d_colbits.alloc(colbits.size() * 4));
    VGA_TRY(d_noc.alloc(node_of_cell.size() * 4));
    VGA_TRY(d_cells.alloc((size_t)std::max<uint32_t>(n, 1) * 4));
    VGA_TRY(d_rowbytes.alloc((size_t)std::max<uint32_t>(n, 1) * 8));
    VGA_TRY(d_counter.alloc(4 * sizeof(uint32_t)));
    VGA_TRY(d_retry.alloc((size_t)std::max<uint32_t>(n, 1) * 4));
    VGA_TRY(d_err.alloc(sizeof(int)));
    cudaStream_t stream = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_rowbits.ptr, rowbits.data(), rowbits.size() * 4, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_colbits.ptr, colbits.data(), colbits.size() * 4, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_noc.ptr, node_of_cell.data(), node_of_cell.size() * 4, cudaMemcpyHostToDevice,
                                   stream));
    if (n) VGA_CHECK_CUDA(cudaMemcpyAsync(d_cells.ptr, cells.data(), (size_t)n * 4, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_counter.ptr, 0, 4 * sizeof(uint32_t), stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_err.ptr, 0, sizeof(int), stream));

    SweepArgs sa{};
    sa.rowbits = d_rowbits.as<uint32_t>();
    sa.colbits = d_colbits.as<uint32_t>();
    sa.W = W;
    sa.H = H;
    sa.words_r = words_r;
    sa.words_c = words_c;
    sa.node_of_cell = d_noc.as<int32_t>();
    sa.cells = d_cells.as<uint32_t>();
    sa.n = n;
    sa.row_bytes = d_rowbytes.as<uint64_t>();
    sa.retry = d_retry.as<uint32_t>();
    sa.retry_count = d_counter.as<uint32_t>() + 2;
    sa.glist_cap = glist_cap;
    sa.words_n = words_n;
    sa.mask_words = mask_words;
    sa.smem_cap = g_sweep_smem_cap;
    sa.err = d_err.as<int>();

    // one launch of the sweep over `count` sources (sources == nullptr: all
    // nodes), interval lists in shared memory or (retries) in global memory
    auto launch = [&](bool write, bool global_lists, const uint32_t *sources, uint32_t count,
                      uint32_t *counter) -> int {
        if (!count) return VGA_OK;
        const size_t smem = (smem_bitmap ? bitmap_smem : 0) + (global_lists ? 0 : list_smem) + mask_smem;
        void (*fn)(SweepArgs);
        if (write) {
            if (global_lists) fn = smem_bitmap ? visibility_sweep_kernel<true, true, true> : visibility_sweep_kernel<true, true, false>;
            else fn = smem_bitmap ? visibility_sweep_kernel<true, false, true> : visibility_sweep_kernel<true, false, false>;
        } else {
            if (global_lists) fn = smem_bitmap ? visibility_sweep_kernel<false, true, true> : visibility_sweep_kernel<false, true, false>;
            else fn = smem_bitmap ? visibility_sweep_kernel<false, false, true> : visibility_sweep_kernel<false, false, false>;
        }
        VGA_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        VGA_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSweepThreads, smem));
        if (per_sm < 1) {
            set_error("visibility sweep: %zu bytes of shared memory do not fit an SM", smem);
            return VGA_EINVAL;
        }
        const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)sms * per_sm, count);
        if (!smem_bitmap) {
            const size_t need = (size_t)grid * words_n * 4;
            if (d_gbitmap.bytes < need) VGA_TRY(d_gbitmap.alloc(need));
            VGA_CHECK_CUDA(cudaMemsetAsync(d_gbitmap.ptr, 0, need, stream));
        }
        if (global_lists) {
            const size_t need = (size_t)grid * kSweepWarps * 2 * glist_cap * sizeof(uint2);
            if (d_glists.bytes < need) VGA_TRY(d_glists.alloc(need));
        }
        SweepArgs a = sa;
        a.sources = sources;
        a.count = count;
        a.next = counter;
        a.gbitmap = d_gbitmap.as<uint32_t>();
        a.glists = d_glists.as<uint2>();
        fn<<<grid, kSweepThreads, smem, stream>>>(a);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        return VGA_OK;
    };

    std::vector<uint64_t> offsets((size_t)n + 1, 0);
    uint32_t n_retry = 0;
    if (n) {
        // count pass; the sources whose lists outgrew shared memory are counted again
        VGA_TRY(launch(false, false, nullptr, n, d_counter.as<uint32_t>()));
        VGA_CHECK_CUDA(cudaMemcpyAsync(&n_retry, sa.retry_count, 4, cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        VGA_TRY(launch(false, true, d_retry.as<uint32_t>(), n_retry, d_counter.as<uint32_t>() + 1));
        std::vector<uint64_t> rb(n);
        int err = 0;
        VGA_CHECK_CUDA(cudaMemcpyAsync(rb.data(), d_rowbytes.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaMemcpyAsync(&err, d_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        if (err) {
            set_error("visibility sweep failed its own checks (code %d)", err);
            return VGA_ECORRUPT;
        }
        for (uint32_t v = 0; v < n; v++) offsets[v + 1] = offsets[v] + rb[v];
    }
    const uint64_t n_bytes = offsets[n];
    DeviceBuffer d_off, d_bytes;
    VGA_TRY(d_off.alloc(((size_t)n + 1) * 8));
    VGA_TRY(d_bytes.alloc(n_bytes + kBytePad));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_off.ptr, offsets.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_bytes.as<uint8_t>() + n_bytes, 0, kBytePad, stream));
    if (n) {
        // write pass: the same split between shared-memory and global lists
        VGA_CHECK_CUDA(cudaMemsetAsync(d_counter.ptr, 0, 2 * sizeof(uint32_t), stream));
        sa.offsets = d_off.as<uint64_t>();
        sa.out = d_bytes.as<uint8_t>();
        VGA_TRY(launch(true, false, nullptr, n, d_counter.as<uint32_t>()));
        VGA_TRY(launch(true, true, d_retry.as<uint32_t>(), n_retry, d_counter.as<uint32_t>() + 1));
        int err = 0;
        VGA_CHECK_CUDA(cudaMemcpyAsync(&err, d_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        if (err) {
            set_error("visibility sweep failed its own checks (code %d)", err);
            return VGA_ECORRUPT;
        }
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    uint64_t *po = d_off.as<uint64_t>();
    uint8_t *pb = d_bytes.as<uint8_t>();
    d_off.release();
    d_bytes.release();
    VGA_TRY(finish_graph_load(n, n_bytes, po, pb, nullptr, stream, out));
    // the builder knows every node's cell: the grouped union groups 2 x 2 blocks
    (*out)->cells.swap(cells);
    (*out)->cells_W = W;
    (*out)->cells_H = H;
    return VGA_OK;
}

int vga_set_visibility_sweep_limits(int smem_list_cap, uint32_t smem_bitmap_nodes) {
    clear_error();
    if (smem_list_cap < 0 || smem_list_cap > kSweepCap) {
        set_error("vga_set_visibility_sweep_limits: list capacity %d outside 0..%d", smem_list_cap, kSweepCap);
        return VGA_EINVAL;
    }
    g_sweep_smem_cap = smem_list_cap ? smem_list_cap : kSweepCap;
    g_sweep_smem_bitmap_nodes = smem_bitmap_nodes;
    return VGA_OK;
}

int vga_visibility_build(int W, int H, const uint8_t *obst, uint64_t *cell_of_node, vga_graph **out) {
    return vga_visibility_build_ordered(W, H, obst, 0, cell_of_node, out);
}

}  // extern "C"
