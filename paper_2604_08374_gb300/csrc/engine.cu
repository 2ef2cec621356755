// engine.cu -- many HyperBall analyses (Algorithm 1) advanced together.
//
// A batch holds jobs (graph, p, d, seed, convergence rule) of any size.  Each
// phase of a pass is one launch for the whole batch:
//   union     a persistent kernel: CTAs claim work items (job, slice, block of
//             W nodes) from an atomic counter, so uneven jobs balance across
//             the GPU; items run in job-major, slice-major order, so the
//             counters being gathered are one job's slice at a time and stay
//             in L2;
//   estimate  one warp per node of every running job (estimator + Eq. sumD);
//   step      one thread per job: pass count, stop rule, flags;
//   finalize  mean depth and ball sizes of the jobs that just stopped.
// The pass loop is either driven from the host (one flag read per pass) or
// captured once as a CUDA graph whose WHILE conditional node repeats the four
// launches until no job is running, with no host round trip at all.
//
// Every job's registers, estimates and outputs are bit-identical to a
// single-graph run of the same job (same device functions, same order of
// floating-point operations per node).
#include <algorithm>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "hb_device.cuh"

namespace vga {



namespace {



// Index of the job whose [start[j], start[j+1]) range holds x.
__device__ __forceinline__ int find_job(const uint64_t *__restrict__ start, int n_jobs, uint64_t x) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_init_kernel(JobDev *jobs, const uint64_t *__restrict__ node_start, int n_jobs,
                                  uint64_t total_nodes) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total_nodes;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const int j = find_job(node_start, n_jobs, x);
        const JobDev &J = jobs[j];
        const uint32_t v = (uint32_t)(x - node_start[j]);
        init_node(J.regs[0], J.n, J.p, J.S, J.seed, v);
        if (J.first) {
            const uint32_t key = node_key(v, J.p, J.seed, false);
            if (J.p <= kKey16MaxP)
                reinterpret_cast<uint16_t *>(J.tab)[v] = KeyFmt<uint16_t>::pack(key);
            else
                reinterpret_cast<uint32_t *>(J.tab)[v] = KeyFmt<uint32_t>::pack(key);
        }
    }
}

// Pass 1 of the jobs in fjobs[0 .. n) (all of precision p, all fresh) as the
// scatter of their nodes' keys, one warp per work item of the concatenated
// work lists (first_pass_item; a per-neighbour job's units are its nodes,
// first_pass_csr); the jobs' union launch skips them in pass 1.
template <class K>
__global__ void __launch_bounds__(kFirstPassWarps * 32) batch_first_pass_kernel(JobDev *jobs,
                                                                               const uint32_t *__restrict__ fjobs,
                                                                               const uint64_t *__restrict__ fstart,
                                                                               int n, int p, int *error) {
    extern __shared__ __align__(16) uint32_t s_cells[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t m = 1u << p;
    uint32_t *cells = s_cells + (uint64_t)wib * (m + 32u);
    const uint64_t total = fstart[n];
    const uint64_t warps = (uint64_t)gridDim.x * kFirstPassWarps;
    for (uint64_t x = (uint64_t)blockIdx.x * kFirstPassWarps + wib; x < total; x += warps) {
        const int k = find_job(fstart, n, x);
        JobDev &J = jobs[fjobs[k]];
        if (J.mode == 2)
            first_pass_item<false, K>(J.items[x - fstart[k]], J.lk, reinterpret_cast<const K *>(J.tab), J.n, J.p,
                                      J.scheme, __ffs(J.S) - 1, 0u, (uint32_t)J.slices, J.regs[1], cells, cells + m,
                                      lane, &J.changed, error);
        else  // per-neighbour job: the work units are its nodes, the scatter decodes the CSR
            first_pass_csr<false, K>(J.off, J.bytes, reinterpret_cast<const K *>(J.tab), (uint32_t)(x - fstart[k]),
                                     J.n, J.p, __ffs(J.S) - 1, 0u, (uint32_t)J.slices, J.regs[1], cells, lane,
                                     &J.changed, error);
    }
}

// initial != 0: c_0 of every job; otherwise pass t = job.t + 1 of running jobs.
__global__ void batch_estimate_kernel(JobDev *jobs, const uint64_t *__restrict__ node_start, int n_jobs,
                                      uint64_t total_nodes, int initial) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t x = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < total_nodes; x += warps) {
        const int j = find_job(node_start, n_jobs, x);
        JobDev &J = jobs[j];
        if (!initial && J.state != 0) continue;
        const int t = initial ? 0 : J.t + 1;
        const double *c_prev = t ? J.c[(t - 1) & 1] : nullptr;
        estimate_node(J.regs[t & 1], J.n, J.p, J.S, t, J.alpha_mm, J.lc, c_prev, J.c[t & 1], J.sum_d, &J.inc,
                      (uint32_t)(x - node_start[j]), lane);
    }
}

// Bounded wait (about a second) for the table items of a slice, published by
// their CTAs (every writer fences before the counter increment).
__device__ __forceinline__ bool wait_tables(const uint32_t *done, uint32_t target) {
    for (uint32_t spin = 0; spin < (1u << 22); spin++) {
        if (*reinterpret_cast<const volatile uint32_t *>(done) >= target) {
            __threadfence();
            return true;
        }
        __nanosleep(256);
    }
    return false;
}

// Persistent union over the running jobs of one group (same union variant,
// same slice width S).  CTAs claim items from the group's queue.  Per job and
// slice the queue holds, in run-aware jobs (RUNS), first the sparse-table
// items (TableShape<S>::B rows each, built by the whole CTA) and then the
// union blocks of kEngineBlock work units (run-aware jobs: a split hub's chunk,
// unioned per node, or a group of kEngineGroupNodes consecutive nodes, unioned
// by the grouped union; per-neighbour jobs: a node), whose warps take the
// block's units one at a time from a shared counter, so that a long unit does
// not hold the others back.  A union block starts once its slice's table
// items are done.  Table items never wait, and every table item of a slice is
// claimed before any of its union blocks, so each wait ends.  Small blocks
// (16 units) over 8-warp CTAs were measured fastest with group units: the
// warps of a CTA wait for each other at every block's end.
// Dynamic shared memory of a run-aware union CTA: the warps' TMA stages, their
// groups' partial rows, then one table item's rows with their halo.
template <int S>
constexpr size_t engine_runs_smem() {
    return (size_t)kEngineWarps * sizeof(LkStage) + (size_t)kEngineWarps * kEngineGroupNodes * S +
           (size_t)TableShape<S>::R * S;
}

template <int S, bool RUNS>
__global__ void __launch_bounds__(kEngineWarps * 32) batch_union_kernel(JobDev *jobs,
                                                                        const uint32_t *__restrict__ gjobs,
                                                                        const uint64_t *__restrict__ item_start,
                                                                        int n_jobs, uint64_t total_items,
                                                                        unsigned long long *counter, int *error) {
    __shared__ uint32_t s_ids[RUNS ? 1 : kEngineWarps][32];
    extern __shared__ __align__(128) unsigned char s_dyn[];
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_next;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    LkStage *s_stage = reinterpret_cast<LkStage *>(s_dyn);
    uint4 *s_part = reinterpret_cast<uint4 *>(s_dyn + (size_t)kEngineWarps * sizeof(LkStage)) +
                    (size_t)wib * kEngineGroupNodes * (S / 16);
    uint8_t *s_tab = s_dyn + (size_t)kEngineWarps * sizeof(LkStage) + (size_t)kEngineWarps * kEngineGroupNodes * S;
    uint32_t phase = 0;  // barrier phases of this warp's TMA stage
    if (RUNS) lk_stage_init(s_stage[wib], lane);
    for (;;) {
        __syncthreads();  // every warp is done with the previous item (and its s_next)
        if (threadIdx.x == 0) {
            s_item = atomicAdd(counter, 1ull);
            s_next = 0;
        }
        __syncthreads();
        const uint64_t item = s_item;
        if (item >= total_items) break;
        const int k = find_job(item_start, n_jobs, item);
        JobDev &J = jobs[gjobs[k]];
        if (J.state != 0) continue;
        if (J.first && J.t == 0) continue;  // pass 1 was the scatter (engine_start)
        const uint32_t ublocks = (J.uunits + kEngineBlock - 1) / kEngineBlock;
        const uint64_t per_slice = (uint64_t)ublocks + (RUNS ? (uint64_t)J.tblocks : 0);
        const uint64_t r = item - item_start[k];
        const uint32_t s = (uint32_t)(r / per_slice);
        uint64_t q = r % per_slice;
        const int t = J.t + 1;
        const uint64_t slice = (uint64_t)s * J.n * S;
        const uint8_t *cur = J.regs[(t - 1) & 1] + slice;
        uint8_t *nxt = J.regs[t & 1] + slice;
        uint8_t *tab = RUNS ? J.tab + (uint64_t)s * table_rows(J.scheme) * J.n * S : nullptr;
        if (RUNS) {
            if (q < (uint64_t)J.tblocks) {
                table_item<S>(cur, tab, J.n, (uint32_t)q * (uint32_t)TableShape<S>::B, s_tab, J.scheme);
                __threadfence();  // every writer publishes its table rows device-wide
                __syncthreads();
                if (threadIdx.x == 0) atomicAdd(J.tab_done + s, 1u);
                continue;
            }
            q -= J.tblocks;
            if (threadIdx.x == 0) {
                // every pass builds the slice's tables, but a scattered pass 1
                s_ok = wait_tables(J.tab_done + s, (uint32_t)(t - J.first) * (uint32_t)J.tblocks);
                if (!s_ok) atomicExch(error, 1);
            }
            __syncthreads();
            if (!s_ok) continue;
        }
        const uint32_t u0 = (uint32_t)q * kEngineBlock;
        const uint32_t u1 = min(u0 + kEngineBlock, J.uunits);
        for (;;) {
            uint32_t x = 0;
            if (lane == 0) x = atomicAdd(&s_next, 1u);
            x = u0 + __shfl_sync(0xffffffffu, x, 0);
            if (x >= u1) break;
            if (RUNS) {
                if (x < J.hub_units)  // a split hub's chunk, per node
                    union_item<S, false>(J.items[x], J.lk, cur, tab, nxt, s_stage[wib], phase, lane, &J.changed,
                                         error, nullptr);
                else
                    union_group<S, false, kEngineGroupNodes>(J.groups[x - J.hub_units], J.grows, J.gcls, cur, tab,
                                                             nxt, s_part, s_stage[wib], phase, lane, &J.changed,
                                                             error, nullptr);
            } else {
                union_node_edges<S>(J.off, J.bytes, cur, nxt, x, s_ids[wib], lane, &J.changed);
            }
        }
    }
}

// One thread per job: close the pass, apply the stop rule, reset the flags and
// the union's item counter; report whether any job still runs.
__global__ void batch_step_kernel(JobDev *jobs, int n_jobs, unsigned long long *counters, int *any_running,
                                  cudaGraphConditionalHandle cond, int use_cond) {
    int running = 0;
    for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) {
        JobDev &J = jobs[j];
        if (J.state == 1) J.state = 2;
        if (J.state == 0) {
            const int t = J.t + 1;
            J.t = t;
            bool stop = J.conv ? (J.inc == 0u) : (J.changed == 0u);
            if (J.d > 0 && t >= J.d) stop = true;
            if (stop) J.state = 1;
            J.changed = 0u;
            J.inc = 0u;
        }
        running |= (J.state == 0);
    }
    running = __syncthreads_or(running);
    if (threadIdx.x < kGroups) counters[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        *any_running = running;
        if (use_cond) cudaGraphSetConditional(cond, running ? 1u : 0u);
    }
}

__global__ void batch_finalize_kernel(JobDev *jobs, const uint64_t *__restrict__ node_start, int n_jobs,
                                      uint64_t total_nodes) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total_nodes;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const int j = find_job(node_start, n_jobs, x);
        const JobDev &J = jobs[j];
        if (J.state != 1) continue;
        finalize_node(J.n, J.comp, J.sum_d, J.c[J.t & 1], J.md, J.ball, (uint32_t)(x - node_start[j]));
    }
}

}  // namespace

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }



// 3/4 of the L2: the persistent union interleaves several jobs' slices, and the
// larger grouped budget of single runs was measured slower on the batch
// workload (0.298 against 0.269 s for the 256 graphs)
uint64_t l2_budget_bytes(int dev) { return union_l2_budget(dev); }

JobLayout job_layout(uint32_t n, int p, int slice_cap, uint64_t budget, int mode, int scheme) {
    JobLayout L;
    L.mode = (mode == 1 || (uint64_t)n > kRunMaxNodes) ? 1 : 2;
    L.scheme = scheme;
    const uint32_t m = 1u << p;
    const uint64_t rows = L.mode == 2 ? (uint64_t)table_rows(scheme) : 1;
    int S = (int)std::min<uint32_t>(m, (uint32_t)(slice_cap > 0 ? slice_cap : 1024));
    while (S > 16 && (uint64_t)S * n * rows > budget) S >>= 1;
    L.S = S;
    L.slices = (int)(m / (uint32_t)S);
    const int B = S >= 1024 ? 16 : 32;  // rows of a table item (TableShape)
    L.tblocks = L.mode == 2 ? (int)((n + B - 1) / B) : 0;
    uint64_t o = 0;
    o = align256(o + (uint64_t)n * m);
    o = align256(o + (uint64_t)n * m);
    o = align256(o + 8ull * n);
    o = align256(o + 8ull * n);
    o = align256(o + 8ull * n);
    if (L.mode == 2) {
        o = align256(o + (uint64_t)table_rows(scheme) * n * m);
        o = align256(o + 4ull * L.slices);
    } else if (p <= kFirstPassMaxP) {
        o = align256(o + 4ull * n);  // the keys of pass 1's scatter
    }
    L.bytes = o;
    return L;
}

int make_jobdev(const vga_graph *g, int p, int d, uint64_t seed, int conv, const JobLayout &L, uint8_t *ws,
                const double *lc, double *md, double *ball, uint32_t hub_lookups, cudaStream_t stream, JobDev *out,
                int group_nodes) {
    JobDev J{};
    const uint64_t n = g->n, m = 1ull << p;
    uint64_t o = 0;
    J.regs[0] = ws + o; o = align256(o + n * m);
    J.regs[1] = ws + o; o = align256(o + n * m);
    J.c[0] = reinterpret_cast<double *>(ws + o); o = align256(o + 8 * n);
    J.c[1] = reinterpret_cast<double *>(ws + o); o = align256(o + 8 * n);
    J.sum_d = reinterpret_cast<double *>(ws + o); o = align256(o + 8 * n);
    if (L.mode == 2) {
        J.tab = ws + o; o = align256(o + (uint64_t)table_rows(L.scheme) * n * m);
        J.tab_done = reinterpret_cast<uint32_t *>(ws + o);
        RunItemList list;
        VGA_TRY(ensure_run_items(g, L.scheme, hub_lookups ? hub_lookups : hub_lookups_auto(g, L.scheme), stream,
                                 &list));
        J.lk = g->lk[L.scheme].d_lk;
        J.scheme = L.scheme;
        J.items = list.items;
        J.units = (uint32_t)list.count;
        if (group_nodes == 1) {  // every work item per node (union_item)
            J.hub_units = J.uunits = (uint32_t)list.count;
        } else {
            const uint32_t hub = hub_lookups ? hub_lookups : hub_lookups_auto(g, L.scheme);
            GroupList groups;
            VGA_TRY(ensure_group_list(g, L.scheme, hub, kEngineGroupNodes, stream, &groups));
            J.groups = groups.items;
            J.grows = groups.rows;
            J.gcls = groups.cls;
            J.hub_units = (uint32_t)list.hub_items;
            J.uunits = (uint32_t)(list.hub_items + groups.count);
        }
    } else {
        J.units = g->n;
        J.uunits = g->n;
        if (p <= kFirstPassMaxP) J.tab = ws + o;  // the keys of pass 1's scatter (job_layout)
    }
    J.first = p <= kFirstPassMaxP ? 1 : 0;
    J.off = g->d_offsets;
    J.bytes = g->d_bytes;
    J.comp = g->d_comp;
    J.lc = lc;
    J.md = md;
    J.ball = ball;
    J.alpha_mm = hll_alpha_host(p) * (double)m * (double)m;
    J.seed = seed;
    J.n = g->n;
    J.p = p;
    J.S = L.S;
    J.slices = L.slices;
    J.d = d;
    J.conv = conv;
    J.mode = L.mode;
    J.tblocks = L.tblocks;
    *out = J;
    return VGA_OK;
}

// Linear-counting tables of p = 4..16 side by side (8 (2^p + 1) bytes each).
uint64_t lc_offset(int p) {
    uint64_t o = 0;
    for (int q = 4; q < p; q++) o = align256(o + 8ull * ((1ull << q) + 1));
    return o;
}
uint64_t lc_all_bytes() { return lc_offset(17); }

int upload_lc_tables(uint8_t *dst, const bool *used, cudaStream_t stream) {
    for (int p = 4; p <= 16; p++) {
        if (used && !used[p]) continue;
        const std::vector<double> &t = lc_table(p);
        VGA_CHECK_CUDA(cudaMemcpyAsync(dst + lc_offset(p), t.data(), 8 * t.size(), cudaMemcpyHostToDevice, stream));
    }
    return VGA_OK;
}



uint64_t engine_arrays_bytes(int cap) {
    const uint64_t c = (uint64_t)std::max(cap, 1);
    return align256(sizeof(JobDev) * c) + align256(8 * (c + 1)) + align256(4 * c) + align256(8 * (c + kGroups)) +
           align256(8 * kGroups) + 256 + align256(4 * c) + align256(8 * (c + kGroups));
}

EngineArrays engine_arrays_at(uint8_t *base, int cap) {
    EngineArrays A;
    const uint64_t c = (uint64_t)std::max(cap, 1);
    uint64_t o = 0;
    A.jobs = reinterpret_cast<JobDev *>(base + o); o = align256(o + sizeof(JobDev) * c);
    A.node_start = reinterpret_cast<uint64_t *>(base + o); o = align256(o + 8 * (c + 1));
    A.gjobs = reinterpret_cast<uint32_t *>(base + o); o = align256(o + 4 * c);
    A.item_start = reinterpret_cast<uint64_t *>(base + o); o = align256(o + 8 * (c + kGroups));
    A.counters = reinterpret_cast<unsigned long long *>(base + o); o = align256(o + 8 * kGroups);
    A.any_running = reinterpret_cast<int *>(base + o);
    A.error = reinterpret_cast<int *>(base + o + 4);
    o += 256;
    A.fjobs = reinterpret_cast<uint32_t *>(base + o); o = align256(o + 4 * c);
    A.fstart = reinterpret_cast<uint64_t *>(base + o);
    A.cap = cap;
    return A;
}

int group_index(int mode, int S) { return (mode == 2 ? 7 : 0) + (31 - __builtin_clz((unsigned)S)) - 4; }

template <int S, bool RUNS>
size_t union_smem() {
    return RUNS ? engine_runs_smem<S>() : 0;
}

// Sets the run-aware union kernels' dynamic shared memory limit once.
int union_smem_attrs() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
#define VGA_A(SS)                                                                                                 \
    if (err == cudaSuccess)                                                                                       \
        err = cudaFuncSetAttribute(batch_union_kernel<SS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                   (int)engine_runs_smem<SS>());
        VGA_A(16) VGA_A(32) VGA_A(64) VGA_A(128) VGA_A(256) VGA_A(512) VGA_A(1024)
#undef VGA_A
    });
    VGA_CHECK_CUDA(err);
    return VGA_OK;
}

template <int S, bool RUNS>
int union_grid(int sms) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_union_kernel<S, RUNS>, kEngineWarps * 32,
                                                  union_smem<S, RUNS>());
    return std::max(1, sms * std::max(1, per_sm));
}

int union_grid_for(int mode, int S, int sms) {
#define VGA_G(SS)                                                                               \
    case SS:                                                                                    \
        return mode == 2 ? union_grid<SS, true>(sms) : union_grid<SS, false>(sms);
    switch (S) {
        VGA_G(16) VGA_G(32) VGA_G(64) VGA_G(128) VGA_G(256) VGA_G(512) VGA_G(1024)
    }
#undef VGA_G
    return sms;
}

// Upload descriptors, the node prefix and the per-group item queues of `jobs`
// (host copies) into A; the host vectors are copied synchronously before the
// function returns.
int engine_upload(const EngineArrays &A, const std::vector<JobDev> &jobs, EngineSet *E, cudaStream_t stream) {
    const int nj = (int)jobs.size();
    if (nj > A.cap) {
        set_error("internal: %d jobs exceed the engine capacity %d", nj, A.cap);
        return VGA_EINVAL;
    }
    VGA_TRY(union_smem_attrs());
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<uint64_t> ns(nj + 1, 0);
    for (int k = 0; k < nj; k++) ns[k + 1] = ns[k] + jobs[k].n;
    std::vector<std::vector<uint32_t>> members(kGroups);
    for (int k = 0; k < nj; k++) members[group_index(jobs[k].mode, jobs[k].S)].push_back((uint32_t)k);
    std::vector<uint32_t> gj;
    std::vector<uint64_t> is;
    E->groups.clear();
    for (int g = 0; g < kGroups; g++) {
        if (members[g].empty()) continue;
        EngineGroup G;
        G.index = g;
        G.mode = jobs[members[g][0]].mode;
        G.S = jobs[members[g][0]].S;
        G.n = (int)members[g].size();
        G.gjob_off = gj.size();
        G.item_off = is.size();
        uint64_t items = 0;
        for (uint32_t k : members[g]) {
            gj.push_back(k);
            is.push_back(items);
            const JobDev &J = jobs[k];
            items += (uint64_t)J.slices * ((uint64_t)((J.uunits + kEngineBlock - 1) / kEngineBlock) +
                                           (J.mode == 2 ? (uint64_t)J.tblocks : 0));
        }
        is.push_back(items);
        G.total_items = items;
        G.grid = (unsigned)union_grid_for(G.mode, G.S, sms);
        E->groups.push_back(G);
    }
    if (nj) VGA_CHECK_CUDA(cudaMemcpyAsync(A.jobs, jobs.data(), sizeof(JobDev) * nj, cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(A.node_start, ns.data(), 8 * (nj + 1), cudaMemcpyHostToDevice, stream));
    if (!gj.empty()) {
        VGA_CHECK_CUDA(cudaMemcpyAsync(A.gjobs, gj.data(), 4 * gj.size(), cudaMemcpyHostToDevice, stream));
        VGA_CHECK_CUDA(cudaMemcpyAsync(A.item_start, is.data(), 8 * is.size(), cudaMemcpyHostToDevice, stream));
    }
    VGA_CHECK_CUDA(cudaMemsetAsync(A.counters, 0, 8 * kGroups, stream));
    VGA_CHECK_CUDA(cudaMemsetAsync(A.any_running, 0, 8, stream));  // running flag and error
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));                  // the host vectors go out of scope
    E->n_jobs = nj;
    E->total_nodes = ns[nj];
    E->grid_nodes = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((E->total_nodes + 255) / 256, (uint64_t)sms * 32));
    E->grid_warps = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((E->total_nodes + 7) / 8, (uint64_t)sms * 64));
    return VGA_OK;
}

// Counters of freshly uploaded jobs: zero their initial registers and sum_d,
// insert every node into its own counter, and estimate c_0.
int engine_start(const EngineArrays &A, const std::vector<JobDev> &jobs, const EngineSet &E, cudaStream_t stream) {
    for (const JobDev &J : jobs) {
        VGA_CHECK_CUDA(cudaMemsetAsync(J.regs[0], 0, (uint64_t)J.n << J.p, stream));
        // split hubs merge into the pass's output by atomic max: it must start below the result
        if (J.mode == 2) VGA_CHECK_CUDA(cudaMemsetAsync(J.regs[1], 0, (uint64_t)J.n << J.p, stream));
        VGA_CHECK_CUDA(cudaMemsetAsync(J.sum_d, 0, 8ull * J.n, stream));
        if (J.mode == 2) VGA_CHECK_CUDA(cudaMemsetAsync(J.tab_done, 0, 4ull * J.slices, stream));
    }
    if (!E.n_jobs) return VGA_OK;
    batch_init_kernel<<<E.grid_nodes, 256, 0, stream>>>(A.jobs, A.node_start, E.n_jobs, E.total_nodes);
    count_launch();
    batch_estimate_kernel<<<E.grid_warps, 256, 0, stream>>>(A.jobs, A.node_start, E.n_jobs, E.total_nodes, 1);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    // pass 1 of the run-aware jobs: the scatter, one launch per precision
    std::vector<uint32_t> fj;
    std::vector<uint64_t> fs;
    struct Launch {
        int p, n;
        size_t job_off, start_off;
    };
    std::vector<Launch> launches;
    for (int p = 4; p <= kFirstPassMaxP; p++) {
        Launch L{p, 0, fj.size(), fs.size()};
        uint64_t items = 0;
        for (size_t k = 0; k < jobs.size(); k++) {
            if (!jobs[k].first || jobs[k].p != p) continue;
            fj.push_back((uint32_t)k);
            fs.push_back(items);
            items += jobs[k].units;
            L.n++;
        }
        if (!L.n) continue;
        fs.push_back(items);
        launches.push_back(L);
    }
    if (launches.empty()) return VGA_OK;
    VGA_CHECK_CUDA(cudaMemcpyAsync(A.fjobs, fj.data(), 4 * fj.size(), cudaMemcpyHostToDevice, stream));
    VGA_CHECK_CUDA(cudaMemcpyAsync(A.fstart, fs.data(), 8 * fs.size(), cudaMemcpyHostToDevice, stream));
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        const int most = kFirstPassWarps * ((1 << kFirstPassMaxP) + 32) * 4;
        attr_err = cudaFuncSetAttribute(batch_first_pass_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        most);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(batch_first_pass_kernel<uint32_t>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
    VGA_CHECK_CUDA(attr_err);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (const Launch &L : launches) {
        const size_t smem = (size_t)kFirstPassWarps * ((1u << L.p) + 32u) * 4u;
        const bool k16 = L.p <= kKey16MaxP;
        int per_sm = 1;
        if (k16)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_first_pass_kernel<uint16_t>,
                                                          kFirstPassWarps * 32, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_first_pass_kernel<uint32_t>,
                                                          kFirstPassWarps * 32, smem);
        const uint64_t items = fs[L.start_off + L.n];
        const unsigned grid = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>((items + kFirstPassWarps - 1) / kFirstPassWarps, (uint64_t)sms * std::max(1, per_sm)));
        if (k16)
            batch_first_pass_kernel<uint16_t><<<grid, kFirstPassWarps * 32, smem, stream>>>(
                A.jobs, A.fjobs + L.job_off, A.fstart + L.start_off, L.n, L.p, A.error);
        else
            batch_first_pass_kernel<uint32_t><<<grid, kFirstPassWarps * 32, smem, stream>>>(
                A.jobs, A.fjobs + L.job_off, A.fstart + L.start_off, L.n, L.p, A.error);
        count_launch();
    }
    VGA_CHECK_CUDA(cudaGetLastError());
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));  // the host vectors go out of scope
    return VGA_OK;
}

template <int S, bool RUNS>
void launch_group(const EngineArrays &A, const EngineGroup &G, cudaStream_t stream, int grid_pct) {
    const unsigned grid = (grid_pct > 0 && grid_pct < 100) ? std::max(1u, G.grid * (unsigned)grid_pct / 100u) : G.grid;
    batch_union_kernel<S, RUNS><<<grid, kEngineWarps * 32, union_smem<S, RUNS>(), stream>>>(A.jobs, A.gjobs + G.gjob_off,
                                                                         A.item_start + G.item_off, G.n,
                                                                         G.total_items, A.counters + G.index, A.error);
}

EngineForks::~EngineForks() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
}

int EngineForks::ensure(int n) {
    while ((int)streams.size() < n) {
        cudaStream_t s = nullptr;
        VGA_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        streams.push_back(s);
    }
    while ((int)events.size() < n + 1) {
        cudaEvent_t e = nullptr;
        VGA_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        events.push_back(e);
    }
    return VGA_OK;
}

int engine_pass(const EngineArrays &A, const EngineSet &E, cudaStream_t stream, cudaGraphConditionalHandle cond,
                int use_cond, int grid_pct, EngineForks *forks) {
    // the union kernels of different slice widths touch different jobs: with
    // forks they run side by side, so one kernel's tail overlaps the others
    const int n_aux = forks ? (int)E.groups.size() - 1 : 0;
    if (n_aux > 0) {
        VGA_TRY(forks->ensure(n_aux));
        VGA_CHECK_CUDA(cudaEventRecord(forks->events[0], stream));
        for (int k = 0; k < n_aux; k++) VGA_CHECK_CUDA(cudaStreamWaitEvent(forks->streams[k], forks->events[0], 0));
    }
    int gi = 0;
    for (const EngineGroup &G : E.groups) {
        cudaStream_t gs = (n_aux > 0 && gi > 0) ? forks->streams[gi - 1] : stream;
        gi++;
#define VGA_G(SS)                                                                         \
    case SS:                                                                              \
        if (G.mode == 2) launch_group<SS, true>(A, G, gs, grid_pct);                      \
        else launch_group<SS, false>(A, G, gs, grid_pct);                                 \
        break;
        switch (G.S) {
            VGA_G(16) VGA_G(32) VGA_G(64) VGA_G(128) VGA_G(256) VGA_G(512) VGA_G(1024)
        }
#undef VGA_G
        count_launch();
    }
    for (int k = 0; k < n_aux; k++) {
        VGA_CHECK_CUDA(cudaEventRecord(forks->events[1 + k], forks->streams[k]));
        VGA_CHECK_CUDA(cudaStreamWaitEvent(stream, forks->events[1 + k], 0));
    }
    batch_estimate_kernel<<<E.grid_warps, 256, 0, stream>>>(A.jobs, A.node_start, E.n_jobs, E.total_nodes, 0);
    count_launch();
    batch_step_kernel<<<1, 256, 0, stream>>>(A.jobs, E.n_jobs, A.counters, A.any_running, cond, use_cond);
    count_launch();
    batch_finalize_kernel<<<E.grid_nodes, 256, 0, stream>>>(A.jobs, A.node_start, E.n_jobs, E.total_nodes);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}

// Capture one pass as the body of a WHILE conditional node and run it until
// no job is running.
int engine_run_graph(const EngineArrays &A, const EngineSet &E, cudaStream_t stream, EngineForks *forks) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    VGA_CHECK_CUDA(cudaGraphCreate(&graph, 0));
    struct GraphGuard {
        cudaGraph_t &g;
        cudaGraphExec_t &e;
        ~GraphGuard() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } guard{graph, exec};
    cudaGraphConditionalHandle cond;
    VGA_CHECK_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams params = {};
    params.type = cudaGraphNodeTypeConditional;
    params.conditional.handle = cond;
    params.conditional.type = cudaGraphCondTypeWhile;
    params.conditional.size = 1;
    cudaGraphNode_t node;
    VGA_CHECK_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params));
    cudaGraph_t body = params.conditional.phGraph_out[0];
    cudaStream_t cap = nullptr;
    VGA_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = VGA_OK;
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        rc = engine_pass(A, E, cap, cond, 1, 100, forks);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &captured);
        if (rc == VGA_OK && e2 != cudaSuccess) {
            set_error("capturing the pass loop failed: %s", cudaGetErrorString(e2));
            rc = VGA_ECUDA;
        }
    } else {
        set_error("cudaStreamBeginCaptureToGraph failed: %s", cudaGetErrorString(e));
        rc = VGA_ECUDA;
    }
    cudaStreamDestroy(cap);
    VGA_TRY(rc);
    VGA_CHECK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    VGA_CHECK_CUDA(cudaGraphLaunch(exec, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    return VGA_OK;
}

namespace {

// ---------------------------------------------------------------------------
// hyperball_run_batch
// ---------------------------------------------------------------------------

struct BatchPlan {
    std::vector<int> idx;          // jobs with N > 0, in batch order
    std::vector<JobLayout> lay;
    std::vector<uint64_t> job_off; // workspace offset of each job's block
    bool lc_used[17] = {false};
    uint64_t off_lc = 0, off_arrays = 0, total = 0;
};

int plan_batch(const vga_job *jobs, int n_jobs, int slice_cap, BatchPlan *B) {
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) {
        set_error("hyperball batch: bad job list");
        return VGA_EINVAL;
    }
    int dev = -1;
    VGA_CHECK_CUDA(cudaGetDevice(&dev));
    const uint64_t budget = l2_budget_bytes(dev);
    uint64_t o = 0;
    for (int i = 0; i < n_jobs; i++) {
        const vga_job &jb = jobs[i];
        if (!jb.graph || jb.p < 4 || jb.p > 16 || (jb.conv_mode != 0 && jb.conv_mode != 1)) {
            set_error("hyperball batch: job %d has a null graph, p outside 4..16 or a bad conv_mode", i);
            return VGA_EINVAL;
        }
        if (jb.graph->device != dev) {
            set_error("hyperball batch: job %d's graph lives on device %d, device %d is current", i,
                      jb.graph->device, dev);
            return VGA_EINVAL;
        }
        if (jb.union_mode < 0 || jb.union_mode > 2) {
            set_error("hyperball batch: job %d has union_mode %d (0, 1 or 2)", i, jb.union_mode);
            return VGA_EINVAL;
        }
        if (jb.graph->n == 0) continue;
        // a job that leaves the variant (and the call the width) automatic takes
        // the autotuner's entry for its degree bucket, if one is installed
        vga_tune_entry te{};
        const bool tabled = tune_table_lookup(jb.graph, &te);
        const int mode = jb.union_mode ? jb.union_mode : (tabled ? te.union_mode : 0);
        const int cap = slice_cap ? slice_cap : (tabled ? te.slice_bytes : 0);
        const JobLayout L = job_layout(jb.graph->n, jb.p, cap, budget, mode, jb.graph->lk_scheme);
        B->idx.push_back(i);
        B->lay.push_back(L);
        B->job_off.push_back(o);
        o = align256(o + L.bytes);
        B->lc_used[jb.p] = true;
    }
    B->off_lc = o;
    o = align256(o + lc_all_bytes());
    B->off_arrays = o;
    o = align256(o + engine_arrays_bytes((int)B->idx.size()));
    B->total = o;
    return VGA_OK;
}

int run_batch(vga_job *jobs, int n_jobs, void *ws_ptr, uint64_t ws_bytes, cudaStream_t stream, int use_graph,
              int slice_cap) {
    BatchPlan B;
    VGA_TRY(plan_batch(jobs, n_jobs, slice_cap, &B));
    DeviceBuffer own;
    if (!ws_ptr) {
        VGA_TRY(own.alloc(B.total));
        ws_ptr = own.ptr;
    } else if (ws_bytes < B.total || (reinterpret_cast<uintptr_t>(ws_ptr) & 255u)) {
        set_error("hyperball batch: workspace of %llu bytes, need %llu (256-byte aligned)",
                  (unsigned long long)ws_bytes, (unsigned long long)B.total);
        return VGA_EINVAL;
    }
    uint8_t *ws = static_cast<uint8_t *>(ws_ptr);
    for (int i = 0; i < n_jobs; i++) {
        jobs[i].iterations = 0;
        jobs[i].status = VGA_OK;
    }
    if (B.idx.empty()) return VGA_OK;
    VGA_TRY(upload_lc_tables(ws + B.off_lc, B.lc_used, stream));
    std::vector<JobDev> host(B.idx.size());
    for (size_t k = 0; k < B.idx.size(); k++) {
        const vga_job &jb = jobs[B.idx[k]];
        vga_tune_entry te{};
        const bool tabled = tune_table_lookup(jb.graph, &te);
        const uint32_t hub = tabled ? (uint32_t)te.hub_lookups : 0u;
        VGA_TRY(make_jobdev(jb.graph, jb.p, jb.d, jb.seed, jb.conv_mode, B.lay[k], ws + B.job_off[k],
                            reinterpret_cast<const double *>(ws + B.off_lc + lc_offset(jb.p)), jb.mean_depth_dev,
                            jb.ball_size_dev, hub, stream, &host[k], tabled ? te.group_nodes : 0));
    }
    const EngineArrays A = engine_arrays_at(ws + B.off_arrays, (int)host.size());
    EngineSet E;
    EngineForks forks;
    VGA_TRY(engine_upload(A, host, &E, stream));
    VGA_TRY(engine_start(A, host, E, stream));
    if (use_graph) {
        VGA_TRY(engine_run_graph(A, E, stream));  // forks measured slower inside the WHILE body
    } else {
        int running = 1;
        while (running) {
            VGA_TRY(engine_pass(A, E, stream, 0, 0, 100, &forks));
            VGA_CHECK_CUDA(cudaMemcpyAsync(&running, A.any_running, sizeof(int), cudaMemcpyDeviceToHost, stream));
            VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
        }
    }
    VGA_CHECK_CUDA(cudaMemcpyAsync(host.data(), A.jobs, sizeof(JobDev) * host.size(), cudaMemcpyDeviceToHost, stream));
    int err = 0;
    VGA_CHECK_CUDA(cudaMemcpyAsync(&err, A.error, sizeof(int), cudaMemcpyDeviceToHost, stream));
    VGA_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (err) {
        set_error("hyperball batch: a union item gave up waiting for its sparse tables");
        return VGA_ETIMEOUT;
    }
    for (size_t k = 0; k < host.size(); k++) jobs[B.idx[k]].iterations = host[k].t;
    return VGA_OK;
}

}  // namespace
}  // namespace vga

using namespace vga;

extern "C" {

int hyperball_batch_workspace_bytes(const vga_job *jobs, int n_jobs, uint64_t *bytes) {
    clear_error();
    if (!bytes) {
        set_error("hyperball_batch_workspace_bytes: null argument");
        return VGA_EINVAL;
    }
    BatchPlan B;
    VGA_TRY(plan_batch(jobs, n_jobs, 0, &B));
    *bytes = B.total;
    return VGA_OK;
}

int hyperball_run_batch(vga_job *jobs, int n_jobs, void *workspace_dev, uint64_t workspace_bytes, void *stream,
                        int use_graph) {
    clear_error();
    return run_batch(jobs, n_jobs, workspace_dev, workspace_bytes, static_cast<cudaStream_t>(stream), use_graph, 0);
}

}  // extern "C"
