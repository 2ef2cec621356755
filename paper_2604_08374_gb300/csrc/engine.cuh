// engine.cuh -- internal interface of the batched HyperBall engine (engine.cu),
// shared with the request server (server.cu).
#pragma once

#include <vector>

#include "vga_common.cuh"

namespace vga {

constexpr int kEngineWarps = 8;
constexpr int kEngineGroupNodes = 4;  // nodes per group of the grouped union in the engine
constexpr uint32_t kEngineBlock = 16;  // work units (hub chunks, node groups) per union block of the queue
constexpr int kGroups = 14;  // union kernels: (per neighbour | per run) x slice width 16..1024

// One analysis as the batched kernels see it (device memory).
struct JobDev {
    const uint64_t *off;
    const uint8_t *bytes;
    const uint32_t *comp;
    const uint32_t *lk;      // run-aware union: the graph's range lookups
    const RunItem *items;    // and its work list (nodes, split hubs' chunks)
    uint8_t *tab;            // table regions, slice s at tab + s * table_rows(scheme) * N * S
    uint32_t *tab_done;      // per slice: table items finished, over all passes
    uint8_t *regs[2];   // slice-major [m/S][N][S]; pass t reads regs[(t-1)&1], writes regs[t&1]
    double *c[2];       // c_t lives in c[t&1]
    double *sum_d;
    const double *lc;
    double *md, *ball;
    double alpha_mm;
    uint64_t seed;
    uint32_t n;
    int p, S, slices, d, conv;
    uint32_t units;         // pass-1 scatter units: work-list entries (mode 2) or nodes (mode 1)
    // mode 2: the grouped union (groups of kGroupAutoNodes consecutive nodes)
    const GroupItem *groups;
    const uint32_t *grows;
    const uint2 *gcls;
    uint32_t hub_units;     // mode 2: split-hub chunks, the first work-list entries, unioned per node
    uint32_t uunits;        // union units per slice: hub chunks then groups (mode 2), or nodes (mode 1)
    int mode;               // 1 one gather per neighbour, 2 per run (sparse tables)
    int tblocks;            // table items per slice (mode 2), TableShape<S>::B rows each
    int scheme;             // table scheme of the lookups (mode 2)
    int first;              // 1: pass 1 is the scatter of the nodes' keys (engine_start; keys in tab)
    uint32_t changed, inc;  // flags of the pass in progress
    int t;                  // passes completed
    int state;              // 0 running, 1 stopped at this step (finalize), 2 done
};

// Per-job union variant, slice width and workspace size (regs0, regs1, c0,
// c1, sum_d, and in mode 2 the sparse tables of every slice and their counters).
struct JobLayout {
    int mode = 2, S = 0, slices = 0, tblocks = 0, scheme = 0;
    uint64_t bytes = 0;
};

// Device arrays the batched kernels read, sized for `cap` jobs.
struct EngineArrays {
    JobDev *jobs = nullptr;
    uint64_t *node_start = nullptr;         // cap + 1: prefix of nodes over all jobs
    uint32_t *gjobs = nullptr;              // cap: job indices ordered by union group
    uint64_t *item_start = nullptr;         // cap + kGroups: per group, prefix of items over its jobs
    unsigned long long *counters = nullptr; // kGroups: the groups' item queues
    int *any_running = nullptr;
    int *error = nullptr;                   // set when a bounded wait gave up
    uint32_t *fjobs = nullptr;              // cap: jobs whose pass 1 is the scatter, grouped by p
    uint64_t *fstart = nullptr;             // cap + 14: per p group, prefix of work items over its jobs
    int cap = 0;
};

// One union kernel launch: the jobs sharing a union variant and slice width.
struct EngineGroup {
    int mode = 1, S = 0, n = 0;
    uint64_t gjob_off = 0, item_off = 0, total_items = 0;
    unsigned grid = 1;
    int index = 0;
};

// Sizes and launch shapes of the job set currently uploaded.
struct EngineSet {
    int n_jobs = 0;
    uint64_t total_nodes = 0;
    unsigned grid_nodes = 1, grid_warps = 1;
    std::vector<EngineGroup> groups;
};

uint64_t align256(uint64_t x);
uint64_t l2_budget_bytes(int dev);
JobLayout job_layout(uint32_t n, int p, int slice_cap, uint64_t budget, int mode, int scheme);
// Device view of one analysis in workspace ws; in mode 2 it builds (on first
// use) the graph's lookups and its work list for hub threshold hub_lookups
// (0 = automatic).
// group_nodes == 1 (a tuned choice) unions every run-aware node per warp;
// otherwise the engine groups kEngineGroupNodes nodes.
int make_jobdev(const vga_graph *g, int p, int d, uint64_t seed, int conv, const JobLayout &L, uint8_t *ws,
                const double *lc, double *md, double *ball, uint32_t hub_lookups, cudaStream_t stream, JobDev *out,
                int group_nodes = 0);
uint64_t lc_offset(int p);
uint64_t lc_all_bytes();
int upload_lc_tables(uint8_t *dst, const bool *used, cudaStream_t stream);
uint64_t engine_arrays_bytes(int cap);
EngineArrays engine_arrays_at(uint8_t *base, int cap);
int engine_upload(const EngineArrays &A, const std::vector<JobDev> &jobs, EngineSet *E, cudaStream_t stream);
int engine_start(const EngineArrays &A, const std::vector<JobDev> &jobs, const EngineSet &E, cudaStream_t stream);
// Auxiliary streams and events with which engine_pass runs the union kernels
// of different slice widths concurrently (fork from the pass's stream, join
// before the estimate): created on first use, destroyed with the object.
struct EngineForks {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // [0]: the fork; [1 + k]: stream k's join
    EngineForks() = default;
    EngineForks(const EngineForks &) = delete;
    EngineForks &operator=(const EngineForks &) = delete;
    ~EngineForks();
    int ensure(int n);  // at least n auxiliary streams
};
// One pass of every uploaded job.  grid_pct < 100 runs the union kernels on
// that share of their usual grid (the server's solo-lane priority).
int engine_pass(const EngineArrays &A, const EngineSet &E, cudaStream_t stream, cudaGraphConditionalHandle cond,
                int use_cond, int grid_pct = 100, EngineForks *forks = nullptr);
int engine_run_graph(const EngineArrays &A, const EngineSet &E, cudaStream_t stream, EngineForks *forks = nullptr);

}  // namespace vga
