// engine.cuh -- internal interface of the batched HyperBall engine (engine.cu),
// shared with the request server (server.cu).
#pragma once

#include <vector>

#include "vga_common.cuh"

namespace vga {

constexpr int kEngineWarps = 8;

// One analysis as the batched kernels see it (device memory).
struct JobDev {
    const uint64_t *off;
    const uint8_t *bytes;
    const uint32_t *comp;
    uint8_t *regs[2];   // slice-major [m/S][N][S]; pass t reads regs[(t-1)&1], writes regs[t&1]
    double *c[2];       // c_t lives in c[t&1]
    double *sum_d;
    const double *lc;
    double *md, *ball;
    double alpha_mm;
    uint64_t seed;
    uint32_t n;
    int p, S, slices, d, conv, blocks;
    uint32_t changed, inc;  // flags of the pass in progress
    int t;                  // passes completed
    int state;              // 0 running, 1 stopped at this step (finalize), 2 done
};

// Per-job slice width and workspace size (regs0, regs1, c0, c1, sum_d).
struct JobLayout {
    int S = 0, slices = 0, blocks = 0;
    uint64_t bytes = 0;
};

// Device arrays the batched kernels read, sized for `cap` jobs.
struct EngineArrays {
    JobDev *jobs = nullptr;
    uint64_t *node_start = nullptr, *item_start = nullptr;
    unsigned long long *counter = nullptr;
    int *any_running = nullptr;
    int cap = 0;
};

// Sizes and launch shapes of the job set currently uploaded.
struct EngineSet {
    int n_jobs = 0;
    uint64_t total_nodes = 0, total_items = 0;
    unsigned grid_nodes = 1, grid_warps = 1, grid_union = 1;
};

uint64_t align256(uint64_t x);
uint64_t l2_budget_bytes(int dev);
JobLayout job_layout(uint32_t n, int p, int slice_cap, uint64_t budget);
JobDev make_jobdev(const vga_graph *g, int p, int d, uint64_t seed, int conv, const JobLayout &L, uint8_t *ws,
                   const double *lc, double *md, double *ball);
uint64_t lc_offset(int p);
uint64_t lc_all_bytes();
int upload_lc_tables(uint8_t *dst, const bool *used, cudaStream_t stream);
uint64_t engine_arrays_bytes(int cap);
EngineArrays engine_arrays_at(uint8_t *base, int cap);
int engine_upload(const EngineArrays &A, const std::vector<JobDev> &jobs, EngineSet *E, cudaStream_t stream);
int engine_start(const EngineArrays &A, const std::vector<JobDev> &jobs, const EngineSet &E, cudaStream_t stream);
int engine_pass(const EngineArrays &A, const EngineSet &E, cudaStream_t stream, cudaGraphConditionalHandle cond,
                int use_cond);
int engine_run_graph(const EngineArrays &A, const EngineSet &E, cudaStream_t stream);

}  // namespace vga
