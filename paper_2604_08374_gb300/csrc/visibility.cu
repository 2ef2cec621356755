// visibility.cu -- visibility graph of an obstacle grid, built on the device
// (Sec. 3.1).  Two free cells see each other iff the closed segment between
// their centres meets no obstacle cell's closed square.  Nodes are the cells of
// the largest 4-connected free component, numbered in raster order (Sec. 3.2),
// so neighbour lists come out sorted and delta-encode into mostly one-byte
// LEB128 varints.
//
// Pipeline: (host) main component and numbering; (device) one warp per
// (source, 32 consecutive targets) walks each segment through the grid and
// ballots the results into an N x ceil(N/32) bit matrix, upper block triangle
// only, then 32 x 32 bit-block transposes fill the lower one; (device) one warp per
// source counts the LEB128 bytes of its row; (host) prefix sum into offsets;
// (device) one warp per source writes the bytes; then the ordinary load path
// validates the stream and derives degrees.
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

__device__ __forceinline__ bool blocked_at(const uint32_t *__restrict__ bits, uint32_t idx) {
    return (__ldg(bits + (idx >> 5)) >> (idx & 31u)) & 1u;
}

// Walk the supercover of the segment between the centres of (x0,y0) and
// (x1,y1): at parameter (2i+1)/(2|dx|) the segment crosses its i-th vertical
// grid line, at (2j+1)/(2|dy|) its j-th horizontal one; equal parameters mean
// it passes through a grid corner, touching the two side cells as well.
__device__ bool segment_clear(const uint32_t *__restrict__ bits, int W, int x0, int y0, int x1, int y1) {
    const int dx = x1 - x0, dy = y1 - y0;
    const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
    const int sx = dx < 0 ? -1 : 1;
    const int sWy = dy < 0 ? -W : W;
    uint32_t idx = (uint32_t)y0 * (uint32_t)W + (uint32_t)x0;
    int i = 0, j = 0;
    int tx = ay, ty = ax;  // (2i+1)|dy| and (2j+1)|dx|: compare crossing parameters without division
    while (i < ax || j < ay) {
        const bool sx_step = (i < ax) && (j == ay || tx <= ty);
        const bool sy_step = (j < ay) && (i == ax || ty <= tx);
        if (sx_step && sy_step) {
            if (blocked_at(bits, idx + sx) || blocked_at(bits, idx + sWy)) return false;
        }
        if (sx_step) {
            idx += sx;
            i++;
            tx += 2 * ay;
        }
        if (sy_step) {
            idx += sWy;
            j++;
            ty += 2 * ax;
        }
        if (blocked_at(bits, idx)) return false;
    }
    return true;
}

// One warp per (source u, word w): lanes test targets 32w .. 32w+31.  The
// relation is symmetric, so only words at or right of u's own 32-column block
// are walked (the upper triangle of 32 x 32 blocks, diagonal blocks in full);
// transpose_blocks_kernel mirrors the rest.
__global__ void visibility_bits_kernel(const uint32_t *__restrict__ obst_bits, const uint32_t *__restrict__ cells,
                                       uint32_t n, int W, uint32_t words, uint32_t *__restrict__ bitmat) {
    const int lane = threadIdx.x & 31;
    const uint32_t u = blockIdx.x;
    const uint32_t w = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= words || w < u / 32u) return;
    const uint32_t t = w * 32 + lane;
    bool vis = false;
    if (t < n && t != u) {
        const uint32_t cu = __ldg(cells + u), ct = __ldg(cells + t);
        vis = segment_clear(obst_bits, W, (int)(cu % (uint32_t)W), (int)(cu / (uint32_t)W), (int)(ct % (uint32_t)W),
                            (int)(ct / (uint32_t)W));
    }
    const uint32_t ballot = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) bitmat[(uint64_t)u * words + w] = ballot;
}

// Mirror block (bi, bj), bj > bi, of the 32 x 32-bit block matrix into (bj, bi):
// lane l holds row bi*32 + l's word bj; ballot j collects bit j of every lane,
// which is row bj*32 + j's word bi.
__global__ void transpose_blocks_kernel(uint32_t n, uint32_t words, uint32_t *__restrict__ bitmat) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // warp -> (bi, bj) with bi < bj < words, row-major over the strict upper triangle
    const uint64_t total = (uint64_t)words * (words - 1) / 2;
    if (warp >= total) return;
    // bi = largest i with i*words - i*(i+1)/2 <= warp; solved by bisection
    uint32_t lo = 0, hi = words - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        const uint64_t start = (uint64_t)mid * words - (uint64_t)mid * (mid + 1) / 2;
        if (start <= warp) lo = mid;
        else hi = mid - 1;
    }
    const uint32_t bi = lo;
    const uint64_t start = (uint64_t)bi * words - (uint64_t)bi * (bi + 1) / 2;
    const uint32_t bj = bi + 1 + (uint32_t)(warp - start);
    const uint32_t row = bi * 32 + lane;
    const uint32_t word = row < n ? bitmat[(uint64_t)row * words + bj] : 0u;
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
        const uint32_t col = __ballot_sync(0xffffffffu, (word >> j) & 1u);
        if (lane == j) mine = col;
    }
    const uint32_t out_row = bj * 32 + lane;
    if (out_row < n) bitmat[(uint64_t)out_row * words + bi] = mine;
}

__device__ __forceinline__ uint32_t varint_len(uint32_t x) {
    return x < (1u << 7) ? 1u : x < (1u << 14) ? 2u : x < (1u << 21) ? 3u : x < (1u << 28) ? 4u : 5u;
}

// One warp per source row; lanes own consecutive words.  The first id of each
// word is encoded relative to the last id of the nearest earlier non-empty
// word (absolute for the row's first id); ids inside a word differ by < 32, so
// their deltas take one byte.  WRITE = false only sums the bytes.
template <bool WRITE>
__global__ void encode_rows_kernel(const uint32_t *__restrict__ bitmat, uint32_t n, uint32_t words,
                                   uint64_t *__restrict__ row_bytes, const uint64_t *__restrict__ offsets,
                                   uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= n) return;
    const uint32_t *row = bitmat + warp * words;
    int64_t prev = -1;   // last id before the current chunk
    uint64_t pos = WRITE ? offsets[warp] : 0;
    uint64_t total = 0;
    for (uint32_t w0 = 0; w0 < words; w0 += 32) {
        const uint32_t wi = w0 + lane;
        const uint32_t word = wi < words ? row[wi] : 0u;
        const int64_t last = word ? (int64_t)wi * 32 + 31 - __clz(word) : -1;
        // exclusive max-scan of `last` over lanes: the previous id for this word
        int64_t incl = last;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o && t > incl) incl = t;
        }
        int64_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = -1;
        if (prev > excl) excl = prev;
        uint32_t nbytes = 0;
        if (word) {
            const uint32_t first = wi * 32 + (__ffs(word) - 1);
            const uint32_t val = excl < 0 ? first : first - (uint32_t)excl;
            nbytes = varint_len(val) + (uint32_t)__popc(word) - 1u;
        }
        // exclusive prefix of byte counts for the write position
        uint32_t s = nbytes;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        const uint32_t chunk_bytes = __shfl_sync(0xffffffffu, s, 31);
        if (WRITE && word) {
            uint64_t q = pos + (s - nbytes);
            uint32_t bitsleft = word;
            int64_t last_id = excl;
            while (bitsleft) {
                const uint32_t id = wi * 32 + (__ffs(bitsleft) - 1);
                bitsleft &= bitsleft - 1u;
                uint32_t x = last_id < 0 ? id : id - (uint32_t)last_id;
                do {
                    uint8_t b = (uint8_t)(x & 0x7Fu);
                    x >>= 7;
                    if (x) b |= 0x80u;
                    out[q++] = b;
                } while (x);
                last_id = id;
            }
        }
        pos += chunk_bytes;
        total += chunk_bytes;
        const int64_t chunk_last = __shfl_sync(0xffffffffu, incl, 31);
        if (chunk_last > prev) prev = chunk_last;
    }
    if (!WRITE && lane == 0) row_bytes[warp] = total;
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
    const uint64_t C = (uint64_t)W * H;
    const uint64_t obst_words = (C + 31) / 32;
    std::vector<uint32_t> bits(obst_words, 0u);
    for (uint64_t c = 0; c < C; c++)
        if (obst[c]) bits[c >> 5] |= 1u << (c & 31);
    const uint32_t words = (n + 31) / 32;
    const uint64_t mat_bytes = (uint64_t)n * words * 4;
    size_t free_b = 0, total_b = 0;
    VGA_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (mat_bytes + (64ull << 20) > free_b) {
        set_error("visibility bit matrix needs %llu bytes, %zu free", (unsigned long long)mat_bytes, free_b);
        return VGA_ENOMEM;
    }
    DeviceBuffer d_bits, d_cells, d_mat, d_rowbytes;
    VGA_TRY(d_bits.alloc(obst_words * 4));
    VGA_TRY(d_cells.alloc((size_t)std::max<uint32_t>(n, 1) * 4));
    VGA_TRY(d_mat.alloc(mat_bytes));
    VGA_TRY(d_rowbytes.alloc((size_t)std::max<uint32_t>(n, 1) * 8));
    cudaStream_t stream = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_bits.ptr, bits.data(), obst_words * 4, cudaMemcpyHostToDevice, stream));
    if (n) VGA_CHECK_CUDA(cudaMemcpyAsync(d_cells.ptr, cells.data(), (size_t)n * 4, cudaMemcpyHostToDevice, stream));
    std::vector<uint64_t> offsets((size_t)n + 1, 0);
    if (n) {
        const int warps = 8;
        const uint32_t wblocks = (words + warps - 1) / warps;
        if (wblocks > 65535u) {
            set_error("graph too large for the builder (%u nodes)", n);
            return VGA_EINVAL;
        }
        dim3 grid(n, wblocks);
        visibility_bits_kernel<<<grid, warps * 32, 0, stream>>>(d_bits.as<uint32_t>(), d_cells.as<uint32_t>(), n, W,
                                                                 words, d_mat.as<uint32_t>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        const uint64_t blocks_upper = (uint64_t)words * (words - 1) / 2;
        if (blocks_upper) {
            transpose_blocks_kernel<<<(unsigned)((blocks_upper + warps - 1) / warps), warps * 32, 0, stream>>>(
                n, words, d_mat.as<uint32_t>());
            count_launch();
            VGA_CHECK_CUDA(cudaGetLastError());
        }
        const unsigned rblocks = (n + warps - 1) / warps;
        encode_rows_kernel<false><<<rblocks, warps * 32, 0, stream>>>(d_mat.as<uint32_t>(), n, words,
                                                                      d_rowbytes.as<uint64_t>(), nullptr, nullptr);
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
        std::vector<uint64_t> rb(n);
        VGA_CHECK_CUDA(cudaMemcpyAsync(rb.data(), d_rowbytes.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, stream));
        VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        for (uint32_t v = 0; v < n; v++) offsets[v + 1] = offsets[v] + rb[v];
    }
    const uint64_t n_bytes = offsets[n];
    DeviceBuffer d_off, d_bytes;
    VGA_TRY(d_off.alloc(((size_t)n + 1) * 8));
    VGA_TRY(d_bytes.alloc(n_bytes + kBytePad));
    VGA_CHECK_CUDA(cudaMemcpyAsync(d_off.ptr, offsets.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(d_bytes.as<uint8_t>() + n_bytes, 0, kBytePad, stream));
    if (n) {
        const int warps = 8;
        const unsigned rblocks = (n + warps - 1) / warps;
        encode_rows_kernel<true><<<rblocks, warps * 32, 0, stream>>>(d_mat.as<uint32_t>(), n, words, nullptr,
                                                                     d_off.as<uint64_t>(), d_bytes.as<uint8_t>());
        count_launch();
        VGA_CHECK_CUDA(cudaGetLastError());
    }
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    d_mat.reset();
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

int vga_visibility_build(int W, int H, const uint8_t *obst, uint64_t *cell_of_node, vga_graph **out) {
    return vga_visibility_build_ordered(W, H, obst, 0, cell_of_node, out);
}

}  // extern "C"
