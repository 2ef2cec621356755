/*
 * vga_hyperball.h -- C ABI of the GB300 HyperBall library for visibility
 * graph analysis.
 *
 * Paper: "City-Scale Visibility Graph Analysis via GPU-Accelerated HyperBall"
 * (arXiv 2604.08374).  The library keeps a visibility graph resident in device
 * memory as the paper's delta-compressed LEB128 CSR (Sec. 3.2) and runs the
 * HyperBall iteration of Algorithm 1 (Sec. 3.3) on it with sm_103a kernels:
 * HyperLogLog counters of m = 2^p uint8 registers, the register-wise union of
 * Eq. hll-union, the HLL estimator, the distance accumulation of Eq. sumD, and
 * Visual Mean Depth MD(v) = sum_d[v] / (N_v - 1).
 *
 * Conventions for every entry point:
 *  - Return value: VGA_OK (0) or a negative vga_status.  On failure
 *    vga_last_error() gives a message for the calling thread; outputs are
 *    unspecified.
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *    Output buffers are caller-owned and must hold the stated element counts.
 *  - "host" pointers are ordinary CPU memory (pinned or pageable); "device"
 *    pointers are CUDA global memory of the current device.
 *  - Node ids are uint32, numbered 0..N-1.  Edges are directed: a visibility
 *    edge u-v appears in both lists, and E = sum of degrees (the paper's edge
 *    counts, Sec. 4.3 edge-density table, count both directions).
 *  - A vga_graph lives on the device that was current when it was loaded; run
 *    it with that device current.
 */
#ifndef VGA_HYPERBALL_H
#define VGA_HYPERBALL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vga_status {
    VGA_OK = 0,
    VGA_EINVAL = -1,    /* bad argument (size, precision, null pointer)        */
    VGA_ENOMEM = -2,    /* device or host allocation failed                    */
    VGA_ECORRUPT = -3,  /* malformed CSR or file                               */
    VGA_ECUDA = -4,     /* a CUDA call failed                                  */
    VGA_ETIMEOUT = -5,  /* a bounded device wait ran out                       */
    VGA_EBUSY = -6,     /* resource budget exhausted, try later                */
    VGA_EIO = -7        /* file could not be read or written                   */
} vga_status;

/* Opaque graph: owns the device-resident compressed CSR. */
typedef struct vga_graph vga_graph;

/* Message describing the last failure on the calling thread ("" if none). */
const char *vga_last_error(void);

/* Library version string. */
const char *vga_version(void);

/* ---------------------------------------------------------------------- */
/* Compressed CSR (Sec. 3.2)                                               */
/* ---------------------------------------------------------------------- */

/*
 * vga_csr_encode -- delta + LEB128 encoding of sorted neighbour lists
 * (Sec. 3.2, "Encoding"): each list's first id is an absolute unsigned
 * LEB128 varint (7-bit groups, least significant first, 0x80 = more bytes
 * follow), every later id the delta (>= 1) from its predecessor.
 *   n        number of nodes.
 *   row_ptr  host, n+1 entries: list of node v is col[row_ptr[v] .. row_ptr[v+1]).
 *   col      host, row_ptr[n] ids, strictly increasing within each list.
 *   offsets  host out, n+1 entries: byte range of node v's list.
 *   bytes    host out or NULL.  With NULL only offsets and *n_bytes are filled
 *            (size query); otherwise it must hold *n_bytes bytes from a size
 *            query.
 *   n_bytes  out: total encoded bytes.
 * Errors: VGA_EINVAL for null pointers or a list that is not strictly
 * increasing.
 */
int vga_csr_encode(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint64_t *offsets,
                   uint8_t *bytes, uint64_t *n_bytes);

/* ---------------------------------------------------------------------- */
/* Graph residency (Sec. 3.2, Sec. 3.4)                                    */
/* ---------------------------------------------------------------------- */

/*
 * vga_graph_load -- copy a compressed CSR to the current device and keep it
 * there (the paper's D1 CompressedCsr: u64 byte offsets, derived u32 degrees,
 * the byte stream).
 *   n_nodes    N >= 0.
 *   offsets    host, N+1 entries, offsets[0] = 0, non-decreasing,
 *              offsets[N] = n_bytes.
 *   bytes      host, n_bytes bytes (may be NULL when n_bytes = 0).
 *   comp_size  host, N entries or NULL: exact component size N_v of each node
 *              (Sec. 3.3); NULL means every node belongs to one component of
 *              size N.
 *   out        receives the graph handle.
 * The byte stream is validated on the device right after the copy: every
 * varint at most 5 bytes and ending inside its node's range, every id < N and
 * different from the node itself, ids strictly increasing.  A malformed graph
 * returns VGA_ECORRUPT (nothing is kept).  Degrees and E are derived here.
 */
int vga_graph_load(uint32_t n_nodes, const uint64_t *offsets, const uint8_t *bytes, uint64_t n_bytes,
                   const uint32_t *comp_size, vga_graph **out);

/* As vga_graph_load, but the offsets and bytes are already in device memory
 * (copied device to device on `stream`, a cudaStream_t or NULL). */
int vga_graph_load_device(uint32_t n_nodes, const uint64_t *offsets_dev, const uint8_t *bytes_dev,
                          uint64_t n_bytes, const uint32_t *comp_size_host, void *stream, vga_graph **out);

/*
 * vga_graph_load_file / vga_graph_save_file -- this library's own binary
 * format (".vgacsr"; the paper's VGACSR03 layout is not published, so this is
 * not byte-compatible with it).  Little-endian: 8-byte magic "VGAHB\0\0\1",
 * u64 N, u64 n_bytes, u64 flags (bit 0: component sizes present), then
 * offsets (N+1 u64), bytes, and N u32 component sizes if flagged.
 * Errors: VGA_EIO (open/read/write), VGA_ECORRUPT (bad header or contents).
 */
int vga_graph_load_file(const char *path, vga_graph **out);
int vga_graph_save_file(const vga_graph *g, const char *path);

/* Release the graph's device memory.  NULL is ignored. */
void vga_graph_free(vga_graph *g);

/* Sizes of a loaded graph: nodes, directed edges, compressed bytes. */
int vga_graph_info(const vga_graph *g, uint32_t *n_nodes, uint64_t *n_edges, uint64_t *n_bytes);

/* Copy the CSR back to host memory: offsets (N+1), bytes (n_bytes), degrees
 * (N).  Any output may be NULL. */
int vga_graph_copy_csr(const vga_graph *g, uint64_t *offsets, uint8_t *bytes, uint32_t *degrees);

/*
 * vga_graph_set_cells -- attach the grid position of every node (Sec. 3.1:
 * node v is the free cell cell_of_node[v] = y * W + x of a W x H grid), as the
 * visibility builder does for the graphs it builds.  The run-aware union then
 * groups nodes by 2 x 2 blocks of cells (vga_tuning.group_nodes = 4, the
 * default), which share more table rows than runs of consecutive ids; the
 * results are the same bit for bit either way.  The graph keeps a host copy
 * (4 bytes a node); cached group lists are dropped.  Any v-to-cell map is
 * accepted as long as every value is below W * H and no two nodes share a
 * cell.  NULL cell_of_node detaches the geometry.  Call it while no analysis
 * runs on the graph.
 *   Errors: VGA_EINVAL for W or H outside 1..16384, a cell out of range or a
 *   cell used twice.
 */
int vga_graph_set_cells(vga_graph *g, int W, int H, const uint64_t *cell_of_node);

/* ---------------------------------------------------------------------- */
/* Visibility graph builder (Sec. 3.1)                                     */
/* ---------------------------------------------------------------------- */

/*
 * vga_visibility_build -- build the visibility graph of an obstacle grid on
 * the device and load it (Sec. 3.1, "Visibility Graph Construction").
 * Rule: two free cells see each other iff the closed segment between their
 * centres meets no obstacle cell's closed square.  Nodes are the cells of the
 * largest 4-connected free component (ties: the component holding the lowest
 * raster index), numbered in row-major raster order (Sec. 3.2).  Only the main
 * component is kept, so N_v = N for every node.
 *   W, H        grid size, 1 <= W, H <= 16384.
 *   obst        host, H*W bytes, row-major (row = y), nonzero = obstacle.
 *   cell_of_node host out or NULL: N entries, raster index y*W+x of each node
 *               (size it W*H to be safe, or query N first with
 *               vga_visibility_count).
 *   out         receives the graph handle.
 * Method: from every source, the 8 octants are swept column by column outwards
 * while a list of the unblocked slope intervals (exact integer fractions,
 * each end open or closed) is kept; a target is visible iff its slope lies in
 * one of them (the diagonal target also needs the cell beside it, whose
 * corner its segment touches, free).  The result equals the pairwise rule
 * above for every pair.  Two passes (count, then write) produce the CSR.
 * Device scratch besides the CSR: obstacle bitmaps (2 x W x H bits with
 * margins), a W*H node-id table and 12 bytes a node; per CTA a node bitmap
 * (in shared memory up to ~800k nodes) and, for sources whose interval lists
 * outgrow shared memory, global lists of max(W, H) + 2 entries per warp.
 * Errors: VGA_EINVAL for bad sizes; VGA_ECORRUPT if the sweep's own checks
 * fail (a visible cell off the component, a list overflow past the proven
 * bound, a count/write mismatch).
 */
int vga_visibility_build(int W, int H, const uint8_t *obst, uint64_t *cell_of_node, vga_graph **out);

/*
 * vga_set_visibility_sweep_limits -- test hook for the builder's two
 * fallbacks: smem_list_cap (1..48, 0 = 48) caps the interval lists kept in
 * shared memory, so that more sources take the global-list retry;
 * smem_bitmap_nodes > 0 keeps the node bitmap in global memory for graphs
 * with more nodes than that (0 = whenever shared memory is too small).
 * Process-wide; both give the same graph as the defaults.
 */
int vga_set_visibility_sweep_limits(int smem_list_cap, uint32_t smem_bitmap_nodes);

/*
 * vga_visibility_build_ordered -- as vga_visibility_build, with the node
 * order chosen: order 0 numbers the main component's cells in row-major
 * raster order, order 1 along the Hilbert curve of the smallest 2^k x 2^k
 * square covering the grid (Sec. 3.2, "Optional Hilbert reordering": nearby
 * cells get nearby ids, which keeps the deltas small; the compressed size
 * stays within about 1 % of raster order).  Raster order makes visible row
 * stretches runs of consecutive ids, which the run-aware union exploits.
 */
int vga_visibility_build_ordered(int W, int H, const uint8_t *obst, int order, uint64_t *cell_of_node,
                                 vga_graph **out);

/* Number of nodes (main-component cells) the builder would produce. */
int vga_visibility_count(int W, int H, const uint8_t *obst, uint32_t *n_nodes);

/* ---------------------------------------------------------------------- */
/* HyperBall (Sec. 3.3, Algorithm 1, Sec. 3.4)                             */
/* ---------------------------------------------------------------------- */

/* Tuning knobs (all 0 = choose automatically). */
typedef struct vga_tuning {
    int slice_bytes;     /* registers per union slice: power of two in [16, min(m, 1024)] */
    int warps_per_cta;   /* union kernel CTA size in warps: 1..16 (0: 4 in mode 2, 8 in 1) */
    int l2_budget_mb;    /* L2 share the auto slice width aims at (default: 3/4 of the L2
                            in mode 2, 60 % in mode 1)                                    */
    int union_mode;      /* 0 auto (= 2), 1 one gather per neighbour, 2 per run of
                            consecutive ids through a sparse table of range maxima; both
                            give the same registers bit for bit.  Mode 2 builds, on a
                            graph's first use, a lookup list held by the graph (4 bytes a
                            lookup, one or a few lookups a run: about 0.66 byte per edge
                            on city graphs with the 5-row table, 0.83 with the 3-row one). */
    int register_bits;   /* 0 or 8: uint8 registers; 4: the paper's packed format (Sec. 3.3,
                            two registers per byte, rho clamped to 15, p >= 5).  4-bit
                            runs are not bit-comparable with 8-bit ones wherever a rho
                            above 15 occurs; they match the same clamp applied alone.      */
    int hub_lookups;     /* mode 2: a node with more range lookups than this is split into
                            chunks of at most this many, each folded by its own warp and
                            merged by a word-wise atomic max (0 = automatic: half of one
                            warp's even share of the lookups, at least 2048)              */
    int table_levels;    /* mode 2: rows per node of a slice's table of range maxima:
                            5 (windows of 1, 2, 4, 8, 16 rows: fewest lookups) or 3 (1, 4,
                            16: lets wider slices fit the L2); 0 = automatic (3 when five
                            rows of 128-byte slices would exceed 5/4 of the L2, the
                            grouped union's budget).  A
                            non-automatic choice builds its own lookup list on first use. */
    int l2_window;       /* 1: during the run, mark the union's table region (mode 2) or
                            register slice (mode 1) persisting in L2 through an access-
                            policy window on the stream, with the process's persisting L2
                            set-aside raised to cover it; both are put back afterwards.
                            0: off (default; the lookup stream is evict-first anyway)      */
    int first_pass;      /* how pass 1 of Eq. hll-union is computed.  Every counter then
                            holds only its own node, so register j of the result is the
                            largest rho among the node's and its neighbours' hashes with
                            index j.  2: that scatter, one launch for all slices (each warp
                            folds the hashes of its node's neighbours, found through the
                            range lookups in mode 2 or by decoding the CSR in mode 1, into
                            m cells of shared memory; p <= 13); 1: the union kernel, like
                            every later pass; 0: automatic (2 wherever allowed).  Same
                            registers bit for bit.                                         */
    int track_changes;   /* at most 32 slices: change tracking.  Each pass records which
                            (node, slice) pairs changed; a node needs the next pass in a
                            slice only if one of its neighbours changed there (otherwise its
                            registers already hold the maximum), which is found before the
                            pass through the range lookups (mode 2) or by decoding the CSR
                            (mode 1), the other nodes keeping their registers.  0: automatic (a pass is tracked when the one before
                            changed fewer than 1 % of the pairs, e.g. the last passes of an
                            unlimited-depth run); 1: off; 2: every pass from the second.
                            Same registers bit for bit.                                    */
    int group_nodes;     /* mode 2: nodes per group of the grouped union.  Consecutive nodes
                            see nearly the same runs, so their lookup lists share entries;
                            each group of this many consecutive (non-hub) nodes gets, on
                            first use, a merged list of its distinct rows sorted by the set
                            of its nodes that need them (held by the graph: 4 bytes a
                            distinct row, about 0.5 byte per edge on city graphs), and one
                            warp gathers each distinct row once.  2, 4 or 8; 1: one node per
                            warp from its own lookups; 0: automatic (4).  Split hubs stay
                            per node.  Same registers bit for bit.                         */
} vga_tuning;

/*
 * vga_set_table_scheme_nodes -- graphs loaded from now on with at least this
 * many nodes get the 3-row table of range maxima (windows of 1, 4 and 16 rows),
 * smaller ones the 5-row table (windows 1..16); 0 restores the automatic
 * choice (3 rows when five rows of 128-byte slices would exceed 3/4 of the L2).
 * Process-wide; the choice fixes which lookups a graph counts at load, and
 * vga_tuning.table_levels can still ask for the other table per run.
 */
int vga_set_table_scheme_nodes(uint32_t nodes);

/*
 * hyperball_run -- Algorithm 1 end to end, host outputs.
 *   g           loaded graph.
 *   p           HLL precision, 4 <= p <= 16; m = 2^p uint8 registers per node.
 *   d           depth limit: run at most d union passes; d <= 0 = unlimited.
 *   seed        hash seed: node v is inserted as splitmix64(v XOR seed); the
 *               top p bits pick the register, rho = leading zeros of the
 *               other 64-p bits + 1 (Sec. 3.3 "Initialisation").
 *   mean_depth  host out, N doubles: MD(v) = sum_d[v] / (N_v - 1), NaN when
 *               N_v <= 1 (Sec. 3.3 "Distance accumulation").
 *   ball_size   host out, N doubles: the estimate c_t[v] of |B(v,t)| after the
 *               last pass run.
 *   iterations  host out or NULL: union passes run.
 * Stopping: after pass t the run ends if t = d or if the pass changed no
 * register anywhere (then every later pass would change nothing and add 0 to
 * sum_d).  The paper's rule max_v(c_t - c_{t-1}) <= 0.5 is available as
 * conv_mode 1 in hyperball_run_dev.
 */
int hyperball_run(const vga_graph *g, int p, int d, uint64_t seed, double *mean_depth, double *ball_size,
                  int *iterations);

/* Bytes of device workspace hyperball_run_dev needs for this graph and p. */
int hyperball_workspace_bytes(const vga_graph *g, int p, uint64_t *bytes);

/*
 * hyperball_run_dev -- as hyperball_run, with device outputs and explicit
 * stream, workspace and tuning.
 *   conv_mode       0: stop at the first pass that changes no register;
 *                   1: the paper's rule (Algorithm 1), stop when
 *                   max_v(c_t - c_{t-1}) <= 0.5.  Both also stop at t = d.
 *   mean_depth_dev  device out, N doubles (may be NULL).
 *   ball_size_dev   device out, N doubles (may be NULL).
 *   iterations      host out or NULL.
 *   workspace_dev   device scratch of at least hyperball_workspace_bytes(),
 *                   256-byte aligned, or NULL to let the library allocate and
 *                   free its own.
 *   stream          cudaStream_t to run on (NULL = legacy default stream).  The
 *                   call returns after the last pass; it synchronises on the
 *                   stream once per pass to read the stop flag.
 *   tuning          NULL or knobs.
 */
int hyperball_run_dev(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth_dev,
                      double *ball_size_dev, int *iterations, void *workspace_dev, uint64_t workspace_bytes,
                      void *stream, const vga_tuning *tuning);

/*
 * hyperball_run_noalloc -- hyperball_run_dev for callers that cannot allocate
 * device memory.  (The paper has no counterpart: this entry point exists for
 * the library's users, not for the method.)
 *
 * Some callers must not call cudaMalloc or cudaFree at run time: code that
 * runs inside a framework whose caching allocator already owns nearly all of
 * the GPU's memory, real-time or long-running services that must not fail or
 * stall after start-up (cudaFree can wait for the whole device to go idle, and
 * cudaMalloc can fail once memory is fragmented or taken), and hosts that budget
 * every device byte up front.  This entry point allocates nothing: its scratch
 * (counters, estimates, flags) is a fixed 64 MiB array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The caller still provides the graph and the device outputs.
 *
 *   Arguments are those of hyperball_run_dev without workspace or tuning;
 *   outputs are device pointers (N doubles each, may be NULL).
 *   The run always uses the per-neighbour union (union_mode 1) with register
 *   slices of min(m, 1024) bytes and 8-bit registers; results are bit for bit
 *   those of hyperball_run_dev.
 *   Size limit: with m = 2^p, s = max(1, m / 1024) slices and A(x) = x rounded
 *   up to a multiple of 256, the run needs
 *       2 A(N m) + 3 A(8 N) + A(8 (m + 1)) + 256
 *       + A(4 N)                      if p <= 13 (first-pass keys)
 *       + A(s N) + 2 A(4 N)           if p <= 15 (change tracking)
 *   bytes, which must not exceed 64 MiB (67,108,864 bytes): about N <= 32,000
 *   nodes at p = 10 or N <= 122,000 at p = 8.  This is the per-neighbour
 *   workspace; hyperball_workspace_bytes sizes the automatic (usually
 *   run-aware, larger) plan and may exceed 64 MiB for a run that fits here.
 *   Larger requests return VGA_EINVAL with a message naming both sizes.
 *   The graph must live on the current device.
 *   Set-up: the first call on each device (and again after the device's
 *   context has been destroyed and re-created, e.g. by cudaDeviceReset) looks
 *   up the array's device address (cudaGetSymbolAddress) with that device
 *   current; make that first call before any stream capture begins.
 *   Sharing: every call on a device uses the same array, and it keeps the last
 *   call's contents; each call clears what must start at zero itself.  Calls
 *   whose work overlaps on the GPU (other streams, other host threads) race on
 *   the array and corrupt each other's results: serialise them.  A call that
 *   fails after launching work waits for that work before it returns.
 */
int hyperball_run_noalloc(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth_dev,
                          double *ball_size_dev, int *iterations, void *stream);

/*
 * hyperball_run_trace -- debug hook for bit-exact checks: as hyperball_run_dev
 * with host outputs, and additionally copies the registers and estimates after
 * every pass.
 *   regs_host   host out or NULL: (max_trace+1) x N x m bytes, node-major
 *               (node v's m registers contiguous); slot 0 holds the initial
 *               counters, slot t the counters after pass t (t <= max_trace).
 *   c_host      host out or NULL: (max_trace+1) x N doubles, c_t likewise.
 */
int hyperball_run_trace(const vga_graph *g, int p, int d, uint64_t seed, int conv_mode, double *mean_depth,
                        double *ball_size, int *iterations, uint8_t *regs_host, double *c_host, int max_trace,
                        const vga_tuning *tuning);


/* ---------------------------------------------------------------------- */
/* Batched analyses                                                        */
/* ---------------------------------------------------------------------- */

/* One analysis of a batch. */
typedef struct vga_job {
    const vga_graph *graph;  /* in: loaded graph on the current device                 */
    int p;                   /* in: HLL precision, 4..16                               */
    int d;                   /* in: depth limit (<= 0: unlimited)                      */
    uint64_t seed;           /* in: hash seed                                          */
    int conv_mode;           /* in: 0 or 1, as in hyperball_run_dev                    */
    int union_mode;          /* in: 0 auto (= 2), 1 per neighbour, 2 per run (vga_tuning) */
    double *mean_depth_dev;  /* out: device, N doubles, or NULL                        */
    double *ball_size_dev;   /* out: device, N doubles, or NULL                        */
    int iterations;          /* out: union passes run                                  */
    int status;              /* out: VGA_OK                                            */
} vga_job;

/* Workspace bytes hyperball_run_batch needs for these jobs. */
int hyperball_batch_workspace_bytes(const vga_job *jobs, int n_jobs, uint64_t *bytes);

/*
 * hyperball_run_batch -- run many analyses (Algorithm 1) together, on graphs
 * of any size and mixed p, d, seed and convergence rule.  Each phase of a pass
 * is one launch for the whole batch: a persistent union kernel whose CTAs take
 * (job, register slice, block of nodes) items from an atomic queue, a batched
 * estimate + Eq. sumD launch, a per-job step (stop rules), and the mean-depth
 * epilogue of the jobs that stopped.  In union mode 2 each (job, slice) is
 * queued as sparse-table items followed by union items, which start once
 * their slice's tables are complete (bounded wait; VGA_ETIMEOUT if it ever
 * gave up).  Per job the results are bit-identical to hyperball_run_dev.
 *   jobs, n_jobs     the batch (jobs with N = 0 are skipped, iterations 0).
 *   workspace_dev    device, >= hyperball_batch_workspace_bytes, 256-byte
 *                    aligned, or NULL to let the library allocate.
 *   stream           cudaStream_t or NULL; the call returns when all jobs are done.
 *   use_graph        0: the host reads a running flag after every pass;
 *                    1: the pass loop is captured once as a CUDA graph with a
 *                    WHILE conditional node and runs with no host round trip.
 */
int hyperball_run_batch(vga_job *jobs, int n_jobs, void *workspace_dev, uint64_t workspace_bytes, void *stream,
                        int use_graph);

/* ---------------------------------------------------------------------- */
/* Serving: a request loop with continuous batching                        */
/* ---------------------------------------------------------------------- */

typedef struct vga_server vga_server;

typedef struct vga_server_config {
    uint64_t hbm_budget_bytes;  /* device bytes requests may hold at once (0: 150 GiB); the
                                   server's memory pool keeps up to this much after requests
                                   finish, for the next ones                                  */
    int max_batch;              /* requests advanced together in the batched lane (0: 256) */
    int solo_nodes;             /* graphs above this many nodes use the solo lane (0: 32768) */
    int lane_priority;          /* 0: lanes equal; 1: solo lane's stream gets the higher
                                   priority; -1: batched lane's does (other values:
                                   VGA_EINVAL)                                                */
    int batched_share;          /* percent of the batched lane's union CTAs kept while a
                                   solo-lane analysis runs, leaving the other SMs to it
                                   (0 or 100: no limit)                                       */
    int reserved[2];
} vga_server_config;

typedef struct vga_server_stats_t {
    uint64_t submitted, completed, queued;
    uint64_t batched_passes;    /* passes the batched lane has run                   */
    uint64_t budget_used, budget_peak;
    uint64_t batched_peak;      /* most requests advanced together in one pass       */
} vga_server_stats_t;

/*
 * vga_server_create -- start a server on the current device.  Analyses
 * (Algorithm 1) of already-loaded graphs are submitted from any thread and run
 * as soon as their device state fits the HBM budget:
 *   - the batched lane (graphs up to solo_nodes nodes) admits waiting requests
 *     between passes and advances all admitted ones together, one pass per
 *     round, through the batched engine (hyperball_run_batch's kernels);
 *     requests join and leave between passes (continuous batching);
 *   - the solo lane runs larger graphs one at a time with hyperball_run_dev's
 *     run-aware union, on its own stream, overlapping the batched lane.
 * Each request's results are bit-identical to running it alone.  Graph
 * memory is the caller's and is not charged to the budget.
 */
int vga_server_create(const vga_server_config *cfg, vga_server **out);

/*
 * vga_server_submit -- queue one analysis.  mean_depth_host and
 * ball_size_host (N doubles each, or NULL) are written when it completes and
 * must stay valid until vga_server_wait returns for it.  The graph must stay
 * loaded until then.  VGA_EBUSY if the request alone exceeds the budget or the
 * server is stopping.
 */
int vga_server_submit(vga_server *s, const vga_graph *g, int p, int d, uint64_t seed, int conv_mode,
                      double *mean_depth_host, double *ball_size_host, uint64_t *request_id);

/*
 * vga_server_wait -- block until the request completes or timeout_s elapses
 * (<= 0: no limit; VGA_ETIMEOUT then).  On completion returns the request's
 * status, passes run, latency (submit to outputs written, seconds) and the
 * part of it spent waiting for admission.  Each id can be waited for once.
 */
int vga_server_wait(vga_server *s, uint64_t request_id, double timeout_s, int *iterations, double *latency_s,
                    double *queued_s);

/* Counters of the server. */
int vga_server_stats(vga_server *s, vga_server_stats_t *out);

/* Finish every submitted request, then stop the lanes and free the server. */
void vga_server_destroy(vga_server *s);

/*
 * vga_metrics -- the closed-form VGA metrics of Sec. 3.3 ("Metric
 * derivation"), from mean depth, the exact component sizes N_v and the
 * degrees of a loaded graph, for every node:
 *   RA = 2 (MD - 1) / (k - 2), k = N_v;
 *   Integration [HH] = 1 / RRA = D_k / RA, with the RRA normaliser
 *     D_k = 2 (k (log2((k+2)/3) - 1) + 1) / ((k-1)(k-2)), the RA of the root of
 *     a diamond-shaped graph of k nodes (Hillier & Hanson; the paper names RRA
 *     but prints no normaliser);
 *   Integration [Tekl] = log2((MD + 2) / 3);
 *   P-value = max(0, 1 - RA);
 *   Point First Moment = MD x deg(v).
 * HH and P-value are NaN when k <= 2 (RA undefined); HH is +inf when MD = 1.
 *   mean_depth_dev  device, N doubles (hyperball_run_dev's output).
 *   out_dev         device out, N x 4 doubles: HH, Tekl, P-value, PFM per node.
 *   stream          cudaStream_t or NULL; the call does not synchronise.
 */
int vga_metrics(const vga_graph *g, const double *mean_depth_dev, double *out_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Measurement (not part of the paper's method)                            */
/* ---------------------------------------------------------------------- */

/* Counters the library keeps for benchmarking.  Kernel launches are always
 * counted; union-kernel launches are timed with CUDA events recorded on the
 * launch stream only while profiling is enabled. */
typedef struct vga_profile {
    uint64_t kernel_launches;     /* library kernels launched since the last reset        */
    uint64_t union_launches;      /* union slices timed (one union kernel, plus the
                                     sparse-table build in mode 2)                        */
    double union_ms;              /* their summed device time                             */
    uint64_t union_edges;         /* neighbour unions they performed (E per slice)        */
    uint64_t union_gather_bytes;  /* register rows gathered x slice bytes, summed: E x S
                                     in mode 1, lookups x S in mode 2                     */
    uint64_t union_hbm_bytes;     /* streamed list bytes (CSR, or 4 x lookups) + 8(N+1)
                                     + 2 x N x slice bytes, summed                        */
    int slice_bytes;              /* slice width of the last timed launch                 */
    int union_mode;               /* union variant of the last timed launch (1 or 2)      */
    int table_rows;               /* rows per node it gathered from: the table scheme's
                                     (mode 2) or 1 (mode 1)                               */
    int reserved;
    uint64_t first_pass_launches; /* first passes computed by the scatter (vga_tuning.
                                     first_pass), timed apart from the union slices       */
    double first_pass_ms;         /* their summed device time                             */
    uint64_t first_pass_edges;    /* neighbour unions they performed (E per launch)       */
    uint64_t tracked_launches;    /* union slices of change-tracked passes (vga_tuning.
                                     track_changes) and the need step before each such
                                     pass, timed apart: their work depends on how many
                                     nodes need it                                        */
    double tracked_ms;            /* their summed device time                             */
} vga_profile;

/* Enable (1) or disable (0) event timing of union launches. */
int vga_profile_enable(int on);
/* Zero every counter. */
int vga_profile_reset(void);
/* Read the counters. */
int vga_profile_read(vga_profile *out);

/*
 * vga_bench_gather -- gather-bandwidth microbenchmark with the union kernel's
 * access pattern: warps gather chunk_bytes-wide slices of pseudo-random rows
 * of a resident_bytes buffer with the same lane mapping and loads in flight as
 * the union kernel, without the LEB128 decode.
 *   resident_bytes  buffer size (rounded down to whole chunks), >= chunk_bytes.
 *   chunk_bytes     power of two in [16, 1024] (the union slice width).
 *   gathers         total chunks gathered (one timed launch after a warm-up).
 *   consumer        1: xor the loaded words (the gather bandwidth itself; sized
 *                   below the L2 this is the L2 gather roofline); 0: fold them
 *                   with the union kernel's bytewise max (its loop's ceiling);
 *                   2: no gather at all -- a coalesced stream of 16-byte loads
 *                   over the buffer (consecutive threads on consecutive words,
 *                   L2-only caching, 4 CTAs of 512 threads per SM), repeated
 *                   until about gathers x chunk_bytes bytes have been read:
 *                   the shape-independent L2 read ceiling of a buffer that
 *                   fits in L2.
 *   stream          cudaStream_t or NULL.
 *   gb_per_s        out: bytes read / kernel time (gathers x chunk_bytes for
 *                   consumers 0 and 1).
 */
int vga_bench_gather(uint64_t resident_bytes, int chunk_bytes, uint64_t gathers, int consumer, void *stream,
                     double *gb_per_s);

/* ---------------------------------------------------------------------- */
/* Register-range shards: one analysis split over several GPUs (or streams)  */
/* by register index.  Eq. hll-union acts on each register independently,   */
/* so shard k keeps only the register slices [s0, s1) of every node's        */
/* counter and runs the union on them alone.  The estimator (Sec. 2.3) needs */
/* all m registers of a node, but only through two sums: the exact integer   */
/* harmonic sum and the zero count.  Each shard writes its part of both for  */
/* every node (its "partial block"); the blocks of all shards, gathered in   */
/* shard order (an all-gather of n_shards x partial_bytes), give every shard */
/* the same c_t, Eq. sumD and mean depth, bit for bit equal to an unsharded  */
/* run.  The stop decision needs the OR of the shards' changed flags.        */
/*                                                                           */
/* Per analysis, on every shard, in lockstep:                                */
/*   vga_shard_start(own) ; all-gather ; vga_shard_estimate(all)   (c_0)     */
/*   repeat: vga_shard_union(own, &changed) ; all-gather ;                   */
/*           vga_shard_estimate(all, &increase) ; OR-reduce changed ;        */
/*           stop as hyperball_run_dev would (changed == 0, or increase == 0 */
/*           under the paper's rule, or t == d)                              */
/*   vga_shard_finalize                                                      */
/* The calls synchronise their stream before returning.  No shard waits on  */
/* another inside a kernel: the exchange is the caller's collective.         */
/* ---------------------------------------------------------------------- */

typedef struct vga_shard vga_shard;

/*
 * vga_shard_create -- shard `shard` of `n_shards` (2 <= n_shards <= the
 * number of register slices, 0 <= shard < n_shards) of the analysis (g, p,
 * seed).  Slices are split as evenly as possible, in order.  `tuning` as for
 * hyperball_run_dev (NULL = automatic; every shard must pass the same).
 * Allocates the shard's device state on the current device; the graph must
 * outlive the shard.
 */
int vga_shard_create(const vga_graph *g, int p, uint64_t seed, int shard, int n_shards, const vga_tuning *tuning,
                     vga_shard **out);

/* Slices held, slice width, and the size of one partial block (256-byte multiple). */
int vga_shard_info(const vga_shard *s, int *slice_first, int *slice_count, int *slice_bytes,
                   uint64_t *partial_bytes);

/* Insert every node into its own counter (Alg. 1) and write this shard's
 * partial block of the initial counters to partial_dev (device, 256-byte aligned). */
int vga_shard_start(vga_shard *s, void *partial_dev, void *stream);

/* One Eq. hll-union pass over this shard's slices, then its partial block of
 * the new counters; *changed (host) = 1 if any of its registers changed. */
int vga_shard_union(vga_shard *s, void *partial_dev, uint32_t *changed, void *stream);

/* c_t of every node from all shards' partial blocks (n_shards consecutive
 * blocks, shard order, device), then Eq. sumD for t >= 1; *increase_flag
 * (host) = 1 if some c_t - c_{t-1} > 0.5 (the paper's rule). */
int vga_shard_estimate(vga_shard *s, const void *all_partials_dev, uint32_t *increase_flag, void *stream);

/* Mean depth and ball size (device, N doubles each, may be NULL), as hyperball_run_dev. */
int vga_shard_finalize(vga_shard *s, double *mean_depth_dev, double *ball_size_dev, void *stream);

void vga_shard_free(vga_shard *s);

/* ---------------------------------------------------------------------- */
/* Autotuner (the paper tunes nothing; its kernel uses one fixed launch      */
/* shape, Sec. 3.4).  Launch choices of the union are picked per degree      */
/* bucket by timing the candidates on the caller's own graphs.               */
/* ---------------------------------------------------------------------- */

/* Tuned launch choices for one degree bucket. */
typedef struct vga_tune_entry {
    int degree_log2;     /* bucket: graphs whose average degree E/N has floor(log2) = this  */
    int union_mode;      /* 1 per neighbour, 2 per run                                       */
    int slice_bytes;     /* slice width; applied as an upper bound, lowered when the slice
                            (and in mode 2 its table of range maxima) would not fit the
                            whole L2 for a larger graph of the bucket                        */
    int warps_per_cta;   /* union CTA size in warps                                          */
    int hub_lookups;     /* mode 2 hub threshold (0 = automatic)                             */
    int p;               /* precision the entry was tuned at                                 */
    double geu_per_s;    /* winner's union throughput on the tuning graph, 1e9 edges/s       */
    uint64_t tuned_edges;/* E of the tuning graph                                            */
    int group_nodes;     /* mode 2 grouped union: nodes per group (0 = automatic, 1 = one node
                            per warp, 2, 4 or 8); the batched engine honours 1 and otherwise
                            groups 4 nodes                                                   */
    int reserved;
} vga_tune_entry;

/*
 * vga_autotune -- time the union's launch choices on the given graphs and
 * return one entry per degree bucket present.
 *   graphs, n_graphs  graphs on the current device (n_graphs >= 1).  Each
 *                     bucket is tuned on its graph with the most edges.
 *   p                 precision to tune at (4..16).
 *   stream            cudaStream_t or NULL.
 *   out, max_out      caller-owned array of entries; *n_out gets the count
 *                     (at most max_out; VGA_EINVAL if more buckets are present).
 *   install           1: also install the result as the process-wide table
 *                     (vga_tune_table_set), 0: only return it.
 * Search per bucket: every union variant and power-of-two slice width that fits
 * the L2 at 8 warps per CTA with the automatic hub threshold; then CTA sizes 4
 * and 16 for the best pair; then, in mode 2, hub thresholds of 1/2 and 1/4 of
 * the automatic one, then group sizes 1, 2 and 8 against the automatic 4.
 * Each candidate runs two union passes (d = 2) twice and
 * keeps its faster run; a run of each variant first builds any lookup list.
 * Every candidate computes the same registers (they differ only in launch shape).
 */
int vga_autotune(const vga_graph *const *graphs, int n_graphs, int p, void *stream, vga_tune_entry *out,
                 int max_out, int *n_out, int install);

/*
 * vga_tune_table_set -- install entries as the process-wide tuning table
 * (copied; n = 0 clears it).  While a table is installed, every analysis whose
 * graph falls in a tabled bucket takes that entry's choices for each tuning
 * field the caller leaves at 0 (hyperball_run, hyperball_run_dev with NULL or
 * partial tuning, hyperball_run_batch and the server; the batched engine uses
 * union_mode and slice_bytes).  hyperball_workspace_bytes follows the table
 * too: query it after the table is set.  Entries with union_mode outside 1..2,
 * slice_bytes not a power of two in [16, 1024] or warps_per_cta outside 0..16
 * give VGA_EINVAL.
 */
int vga_tune_table_set(const vga_tune_entry *entries, int n);

/* Copy the installed table into out (at most max_out entries); *n_out gets its size. */
int vga_tune_table_get(vga_tune_entry *out, int max_out, int *n_out);

#ifdef __cplusplus
}
#endif

#endif /* VGA_HYPERBALL_H */
