// vga_graph.cu -- graph residency: the delta-compressed LEB128 CSR of Sec. 3.2
// kept in device memory, its on-device validation, the host encoder and the
// library's file format.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "runs.cuh"

namespace vga {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// One warp per node v0 .. v1-1: decode its byte range 512 bytes at a time
// (scan_window16) and check every rule of the format.  Writes the degree and the number of range
// lookups the run-aware union will need (runs.cuh), and folds E, the maximum
// degree and the lowest bad node id into global counters.
__global__ void validate_kernel(const uint64_t *__restrict__ off, const uint8_t *__restrict__ bytes, uint32_t n,
                                uint32_t v0, uint32_t v1, int scheme, uint32_t *__restrict__ degree,
                                uint32_t *__restrict__ lk_count, unsigned long long *__restrict__ edge_total,
                                uint32_t *__restrict__ max_degree, uint32_t *__restrict__ bad_node) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)v0 + (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= v1) return;
    const uint32_t v = (uint32_t)warp;
    uint64_t pos = off[v];
    const uint64_t end = off[v + 1];
    uint64_t base = 0;
    uint32_t cnt = 0;
    bool ok = true;
    RunCarry rc;
    while (pos < end) {
        const Window16 W = scan_window16<true>(bytes, pos, end, base, cnt == 0, n, v, scheme, rc, lane);
        if (W.count == 0 || W.fail) {  // a varint runs past the node's range, or a rule is broken
            ok = false;
            break;
        }
        cnt += (uint32_t)W.count;
        pos += W.advance;
    }
    finish_runs(rc, scheme);
    if (lane == 0) {
        degree[v] = ok ? cnt : 0;
        lk_count[v] = ok ? (uint32_t)rc.out : 0u;
        if (!ok) atomicMin(bad_node, v);
        atomicAdd(edge_total, (unsigned long long)cnt);
        atomicMax(max_degree, cnt);
    }
}

static int launch_validate(const uint64_t *d_offsets, const uint8_t *d_bytes, uint32_t n, uint32_t v0, uint32_t v1,
                           int scheme, uint32_t *degree, uint32_t *lk_count, unsigned long long *d_edges,
                           uint32_t *d_maxdeg, uint32_t *d_bad, cudaStream_t stream) {
    if (v1 <= v0) return VGA_OK;
    const int warps = 8;
    const uint64_t blocks = ((uint64_t)(v1 - v0) + warps - 1) / warps;
    validate_kernel<<<(unsigned)blocks, warps * 32, 0, stream>>>(d_offsets, d_bytes, n, v0, v1, scheme, degree,
                                                                  lk_count, d_edges, d_maxdeg, d_bad);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

// Validation of a freshly copied CSR; with h_bytes given, the byte stream is
// also copied here, in chunks, and each chunk's complete nodes are validated
// on a second stream while the next chunk is in flight.
int finish_graph_load(uint32_t n, uint64_t n_bytes, uint64_t *d_offsets, uint8_t *d_bytes, const uint32_t *comp_host,
                      cudaStream_t stream, vga_graph **out, const uint64_t *h_offsets, const uint8_t *h_bytes) {
    DeviceBuffer offsets, bytes, degree, comp, counters, lk_count;
    offsets.ptr = d_offsets;
    bytes.ptr = d_bytes;
    int device = 0;
    VGA_CHECK_CUDA(cudaGetDevice(&device));
    const int scheme = table_scheme_auto(n, device);  // the lookups counted during validation
    VGA_TRY(degree.alloc(sizeof(uint32_t) * (size_t)(n ? n : 1)));
    VGA_TRY(lk_count.alloc(sizeof(uint32_t) * (size_t)(n ? n : 1)));
    if (comp_host) {
        VGA_TRY(comp.alloc(sizeof(uint32_t) * (size_t)n));
        VGA_CHECK_CUDA(cudaMemcpyAsync(comp.ptr, comp_host, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice,
                                       stream));
    }
    VGA_TRY(counters.alloc(64));
    VGA_CHECK_CUDA(cudaMemsetAsync(counters.ptr, 0, 64, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(counters.as<uint8_t>() + 12, 0xFF, 4, stream));  // bad_node = UINT32_MAX
    unsigned long long *d_edges = counters.as<unsigned long long>();
    uint32_t *d_maxdeg = reinterpret_cast<uint32_t *>(counters.as<uint8_t>() + 8);
    uint32_t *d_bad = reinterpret_cast<uint32_t *>(counters.as<uint8_t>() + 12);
    if (h_bytes && n_bytes > 0) {
        constexpr uint64_t kChunk = 256ull << 20;
        cudaStream_t vs = nullptr;
        cudaEvent_t ev = nullptr;
        VGA_CHECK_CUDA(cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking));
        struct Cleanup {
            cudaStream_t &s;
            cudaEvent_t &e;
            ~Cleanup() {
                if (e) cudaEventDestroy(e);
                if (s) cudaStreamDestroy(s);
            }
        } cleanup{vs, ev};
        VGA_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        VGA_CHECK_CUDA(cudaEventRecord(ev, stream));  // offsets, pad and counters are set
        VGA_CHECK_CUDA(cudaStreamWaitEvent(vs, ev, 0));
        uint32_t done = 0;
        for (uint64_t c0 = 0; c0 < n_bytes; c0 += kChunk) {
            const uint64_t c1 = std::min(c0 + kChunk, n_bytes);
            VGA_CHECK_CUDA(cudaMemcpyAsync(d_bytes + c0, h_bytes + c0, c1 - c0, cudaMemcpyHostToDevice, stream));
            VGA_CHECK_CUDA(cudaEventRecord(ev, stream));
            VGA_CHECK_CUDA(cudaStreamWaitEvent(vs, ev, 0));
            // nodes whose byte range ends by c1
            const uint32_t upto = c1 == n_bytes ? n
                                                : (uint32_t)(std::upper_bound(h_offsets + 1, h_offsets + n + 1, c1) -
                                                             (h_offsets + 1));
            VGA_TRY(launch_validate(d_offsets, d_bytes, n, done, upto, scheme, degree.as<uint32_t>(),
                                    lk_count.as<uint32_t>(), d_edges, d_maxdeg, d_bad, vs));
            done = std::max(done, upto);
        }
        VGA_CHECK_CUDA(cudaEventRecord(ev, vs));
        VGA_CHECK_CUDA(cudaStreamWaitEvent(stream, ev, 0));
    } else if (n > 0) {
        VGA_TRY(launch_validate(d_offsets, d_bytes, n, 0, n, scheme, degree.as<uint32_t>(), lk_count.as<uint32_t>(),
                                d_edges, d_maxdeg, d_bad, stream));
    }
    uint8_t host_counters[16];
    std::vector<uint32_t> h_cnt(n);
    VGA_CHECK_CUDA(cudaMemcpyAsync(host_counters, counters.ptr, 16, cudaMemcpyDeviceToHost, stream));
    if (n) VGA_CHECK_CUDA(cudaMemcpyAsync(h_cnt.data(), lk_count.ptr, 4 * (size_t)n, cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    uint64_t edges;
    uint32_t maxdeg, bad;
    memcpy(&edges, host_counters, 8);
    memcpy(&maxdeg, host_counters + 8, 4);
    memcpy(&bad, host_counters + 12, 4);
    if (bad != 0xFFFFFFFFu) {
        set_error("malformed CSR: the byte range of node %u breaks the LEB128 delta format", bad);
        return VGA_ECORRUPT;
    }
    vga_graph *g = new (std::nothrow) vga_graph;
    if (!g) {
        set_error("out of host memory");
        return VGA_ENOMEM;
    }
    cudaGetDevice(&g->device);
    g->n = n;
    g->n_bytes = n_bytes;
    g->n_edges = edges;
    g->max_degree = maxdeg;
    g->d_offsets = static_cast<uint64_t *>(offsets.release());
    g->d_bytes = static_cast<uint8_t *>(bytes.release());
    g->d_degree = static_cast<uint32_t *>(degree.release());
    g->d_comp = static_cast<uint32_t *>(comp.release());
    // offsets of the run-aware union's lookups (the list itself is built on first use)
    g->lk_scheme = scheme;
    vga_graph::RunLookups &L = g->lk[scheme];
    L.h_off.assign((size_t)n + 1, 0);
    for (uint32_t v = 0; v < n; v++) L.h_off[v + 1] = L.h_off[v] + h_cnt[v];
    L.total = L.h_off[n];
    *out = g;
    return VGA_OK;
}

static int check_offsets(uint32_t n, const uint64_t *offsets, uint64_t n_bytes) {
    if (offsets[0] != 0 || offsets[n] != n_bytes) {
        set_error("offsets[0] must be 0 and offsets[N] must equal n_bytes (got %llu, %llu vs %llu)",
                  (unsigned long long)offsets[0], (unsigned long long)offsets[n], (unsigned long long)n_bytes);
        return VGA_ECORRUPT;
    }
    for (uint32_t v = 0; v < n; v++)
        if (offsets[v + 1] < offsets[v]) {
            set_error("offsets decrease at node %u", v);
            return VGA_ECORRUPT;
        }
    return VGA_OK;
}

static int check_comp(uint32_t n, const uint32_t *comp) {
    if (!comp) return VGA_OK;
    for (uint32_t v = 0; v < n; v++)
        if (comp[v] == 0) {
            set_error("component size of node %u is 0", v);
            return VGA_EINVAL;
        }
    return VGA_OK;
}

}  // namespace vga

using namespace vga;

extern "C" {

const char *vga_last_error(void) { return g_err; }

const char *vga_version(void) { return "vga-hyperball 0.1 (sm_103a)"; }

int vga_csr_encode(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint64_t *offsets, uint8_t *bytes,
                   uint64_t *n_bytes) {
    clear_error();
    if (!row_ptr || !offsets || !n_bytes || (!col && row_ptr[n] > 0)) {
        set_error("vga_csr_encode: null argument");
        return VGA_EINVAL;
    }
    uint64_t pos = 0;
    for (uint32_t v = 0; v < n; v++) {
        offsets[v] = pos;
        uint32_t prev = 0;
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            const uint32_t id = col[e];
            if (e > row_ptr[v] && id <= prev) {
                set_error("vga_csr_encode: list of node %u is not strictly increasing", v);
                return VGA_EINVAL;
            }
            uint32_t x = (e == row_ptr[v]) ? id : id - prev;
            do {  // 7 bits per byte, low group first; 0x80 flags a continuation
                uint8_t byte = (uint8_t)(x & 0x7Fu);
                x >>= 7;
                if (x) byte |= 0x80u;
                if (bytes) bytes[pos] = byte;
                pos++;
            } while (x);
            prev = id;
        }
    }
    offsets[n] = pos;
    *n_bytes = pos;
    return VGA_OK;
}

int vga_graph_load_device(uint32_t n, const uint64_t *offsets_dev, const uint8_t *bytes_dev, uint64_t n_bytes,
                          const uint32_t *comp_size, void *stream_ptr, vga_graph **out) {
    clear_error();
    if (!out || !offsets_dev || (n_bytes > 0 && !bytes_dev)) {
        set_error("vga_graph_load_device: null argument");
        return VGA_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    std::vector<uint64_t> h_off((size_t)n + 1);
    VGA_CHECK_CUDA(cudaMemcpyAsync(h_off.data(), offsets_dev, sizeof(uint64_t) * ((size_t)n + 1),
                                   cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    VGA_TRY(check_offsets(n, h_off.data(), n_bytes));
    VGA_TRY(check_comp(n, comp_size));
    DeviceBuffer off, bytes;
    VGA_TRY(off.alloc(sizeof(uint64_t) * ((size_t)n + 1)));
    VGA_TRY(bytes.alloc(n_bytes + kBytePad));
    VGA_CHECK_CUDA(cudaMemcpyAsync(off.ptr, offsets_dev, sizeof(uint64_t) * ((size_t)n + 1),
                                   cudaMemcpyDeviceToDevice, stream));
    if (n_bytes)
        VGA_CHECK_CUDA(cudaMemcpyAsync(bytes.ptr, bytes_dev, n_bytes, cudaMemcpyDeviceToDevice, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(bytes.as<uint8_t>() + n_bytes, 0, kBytePad, stream));
    uint64_t *po = off.as<uint64_t>();
    uint8_t *pb = bytes.as<uint8_t>();
    off.release();
    bytes.release();
    return finish_graph_load(n, n_bytes, po, pb, comp_size, stream, out);
}

int vga_graph_load(uint32_t n, const uint64_t *offsets, const uint8_t *bytes_host, uint64_t n_bytes,
                   const uint32_t *comp_size, vga_graph **out) {
    clear_error();
    if (!out || !offsets || (n_bytes > 0 && !bytes_host)) {
        set_error("vga_graph_load: null argument");
        return VGA_EINVAL;
    }
    VGA_TRY(check_offsets(n, offsets, n_bytes));
    VGA_TRY(check_comp(n, comp_size));
    DeviceBuffer off, bytes;
    VGA_TRY(off.alloc(sizeof(uint64_t) * ((size_t)n + 1)));
    VGA_TRY(bytes.alloc(n_bytes + kBytePad));
    cudaStream_t stream = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(off.ptr, offsets, sizeof(uint64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                                   stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(bytes.as<uint8_t>() + n_bytes, 0, kBytePad, stream));
    uint64_t *po = off.as<uint64_t>();
    uint8_t *pb = bytes.as<uint8_t>();
    off.release();
    bytes.release();
    // the byte stream is copied in chunks, overlapped with validation
    return finish_graph_load(n, n_bytes, po, pb, comp_size, stream, out, offsets, bytes_host);
}

void vga_graph_free(vga_graph *g) {
    if (!g) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    cudaFree(g->d_offsets);
    cudaFree(g->d_bytes);
    cudaFree(g->d_degree);
    if (g->d_comp) cudaFree(g->d_comp);
    for (const vga_graph::RunLookups &L : g->lk) {
        if (L.d_off) cudaFree(L.d_off);
        if (L.d_lk) cudaFree(L.d_lk);
        for (const vga_graph::RunItemSet &r : L.items) cudaFree(r.d_items);
        for (const vga_graph::RunLookups::GroupSet &gs : L.groups) {
            cudaFree(gs.d_items);
            cudaFree(gs.d_rows);
            cudaFree(gs.d_cls);
        }
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    delete g;
}

int vga_graph_set_cells(vga_graph *g, int W, int H, const uint64_t *cell_of_node) {
    clear_error();
    if (!g) {
        set_error("vga_graph_set_cells: null graph");
        return VGA_EINVAL;
    }
    std::vector<uint32_t> cells;
    if (cell_of_node) {
        if (W < 1 || H < 1 || W > 16384 || H > 16384) {
            set_error("vga_graph_set_cells: W = %d, H = %d outside 1..16384", W, H);
            return VGA_EINVAL;
        }
        const uint64_t C = (uint64_t)W * H;
        std::vector<uint8_t> used(C, 0);
        cells.resize(g->n);
        for (uint32_t v = 0; v < g->n; v++) {
            const uint64_t c = cell_of_node[v];
            if (c >= C || used[c]) {
                set_error("vga_graph_set_cells: node %u has cell %llu, outside the %d x %d grid or used twice", v,
                          (unsigned long long)c, W, H);
                return VGA_EINVAL;
            }
            used[c] = 1;
            cells[v] = (uint32_t)c;
        }
    }
    std::lock_guard<std::mutex> lock(g->lk_mu);
    g->cells.swap(cells);
    g->cells_W = cell_of_node ? W : 0;
    g->cells_H = cell_of_node ? H : 0;
    // the group lists were formed from the old geometry
    for (vga_graph::RunLookups &L : g->lk) {
        for (const vga_graph::RunLookups::GroupSet &gs : L.groups) {
            cudaFree(gs.d_items);
            cudaFree(gs.d_rows);
            cudaFree(gs.d_cls);
        }
        L.groups.clear();
    }
    return VGA_OK;
}

int vga_graph_info(const vga_graph *g, uint32_t *n_nodes, uint64_t *n_edges, uint64_t *n_bytes) {
    clear_error();
    if (!g) {
        set_error("vga_graph_info: null graph");
        return VGA_EINVAL;
    }
    if (n_nodes) *n_nodes = g->n;
    if (n_edges) *n_edges = g->n_edges;
    if (n_bytes) *n_bytes = g->n_bytes;
    return VGA_OK;
}

int vga_graph_copy_csr(const vga_graph *g, uint64_t *offsets, uint8_t *bytes, uint32_t *degrees) {
    clear_error();
    if (!g) {
        set_error("vga_graph_copy_csr: null graph");
        return VGA_EINVAL;
    }
    if (offsets)
        VGA_CHECK_CUDA(cudaMemcpy(offsets, g->d_offsets, sizeof(uint64_t) * ((size_t)g->n + 1),
                                  cudaMemcpyDeviceToHost));
    if (bytes && g->n_bytes) VGA_CHECK_CUDA(cudaMemcpy(bytes, g->d_bytes, g->n_bytes, cudaMemcpyDeviceToHost));
    if (degrees && g->n)
        VGA_CHECK_CUDA(cudaMemcpy(degrees, g->d_degree, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
    return VGA_OK;
}

static const char kMagic[8] = {'V', 'G', 'A', 'H', 'B', 0, 0, 1};

int vga_graph_save_file(const vga_graph *g, const char *path) {
    clear_error();
    if (!g || !path) {
        set_error("vga_graph_save_file: null argument");
        return VGA_EINVAL;
    }
    std::vector<uint64_t> off((size_t)g->n + 1);
    std::vector<uint8_t> bytes((size_t)g->n_bytes);
    std::vector<uint32_t> comp;
    VGA_TRY(vga_graph_copy_csr(g, off.data(), bytes.data(), nullptr));
    uint64_t flags = 0;
    if (g->d_comp) {
        flags |= 1;
        comp.resize(g->n);
        VGA_CHECK_CUDA(cudaMemcpy(comp.data(), g->d_comp, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
    }
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return VGA_EIO;
    }
    uint64_t hdr[3] = {g->n, g->n_bytes, flags};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, 8, 3, f) == 3 &&
              fwrite(off.data(), 8, off.size(), f) == off.size() &&
              fwrite(bytes.data(), 1, bytes.size(), f) == bytes.size() &&
              (comp.empty() || fwrite(comp.data(), 4, comp.size(), f) == comp.size());
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return VGA_EIO;
    }
    return VGA_OK;
}

int vga_graph_load_file(const char *path, vga_graph **out) {
    clear_error();
    if (!path || !out) {
        set_error("vga_graph_load_file: null argument");
        return VGA_EINVAL;
    }
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return VGA_EIO;
    }
    char magic[8];
    uint64_t hdr[3];
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kMagic, 8) != 0 || fread(hdr, 8, 3, f) != 3 ||
        hdr[0] > 0xFFFFFFFFull || (hdr[2] & ~1ull) != 0) {
        fclose(f);
        set_error("%s is not a vga-hyperball graph file", path);
        return VGA_ECORRUPT;
    }
    const uint32_t n = (uint32_t)hdr[0];
    std::vector<uint64_t> off((size_t)n + 1);
    std::vector<uint8_t> bytes((size_t)hdr[1]);
    std::vector<uint32_t> comp((hdr[2] & 1) ? n : 0);
    bool ok = fread(off.data(), 8, off.size(), f) == off.size() &&
              fread(bytes.data(), 1, bytes.size(), f) == bytes.size() &&
              (comp.empty() || fread(comp.data(), 4, comp.size(), f) == comp.size());
    fclose(f);
    if (!ok) {
        set_error("%s is truncated", path);
        return VGA_ECORRUPT;
    }
    return vga_graph_load(n, off.data(), bytes.data(), hdr[1], comp.empty() ? nullptr : comp.data(), out);
}

}  // extern "C"
