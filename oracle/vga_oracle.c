/*
 * vga_oracle.c -- CPU oracle for GPU HyperBall over a visibility graph.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library under
 * paper_2604_08374_gb300/; neither side includes or links the other.
 *
 * Paper: "City-Scale Visibility Graph Analysis via GPU-Accelerated HyperBall"
 * (arXiv 2604.08374).  Each function names the passage it follows.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread -lm
 * (-ffp-contract=off matters: gcc contracts a*b+c into FMA by default on
 * aarch64, and the accumulation of Eq. sumD must round each step.)
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - Visibility (Sec. 3.1): two free cells see each other iff the closed
 *    segment between their centres meets no obstacle cell's closed square.
 *  - Node ids (Sec. 3.2): cells of the main component in row-major raster
 *    order.
 *  - CSR (Sec. 3.2): the first neighbour is an absolute unsigned LEB128
 *    varint, each later one the (>= 1) delta from the previous neighbour.
 *  - Hash (Sec. 3.3): SplitMix64 with its state increment
 *    (z = x + 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds and
 *    the final xor-shift), applied to (node id XOR seed).  The top p bits of
 *    the hash are the register index; rho = leading zeros of the remaining
 *    64-p bits + 1 (65-p when they are all zero).
 *  - Estimator (Sec. 2.3, Sec. 3.3): the Flajolet et al. harmonic-mean
 *    estimator with alpha_m, and linear counting m*ln(m/V) when the raw
 *    estimate is <= 2.5m and V > 0 zero registers remain.  The harmonic sum
 *    is formed exactly as an integer and rounded once to double.
 *  - Convergence (Alg. 1): mode 0 stops at the first pass that changes no
 *    register anywhere; mode 1 is the paper's rule, max_v(c_t - c_{t-1})
 *    <= 0.5.  Both also stop after d passes when d > 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Visibility (Sec. 3.1).  obst is an H x W row-major array, 1 = obstacle.   */
/* ------------------------------------------------------------------------ */

static int is_obst(const uint8_t *obst, int W, int H, int x, int y) {
    if (x < 0 || y < 0 || x >= W || y >= H) return 1; /* never reached for in-grid endpoints */
    return obst[(int64_t)y * W + x] != 0;
}

/* Brute force: does the closed segment between the centres of cells (x1,y1)
 * and (x2,y2) meet the closed square of cell (i,j)?  Doubled coordinates make
 * every quantity an integer: the centre of (x,y) is (2x+1, 2y+1) and the
 * square of (i,j) is [2i, 2i+2] x [2j, 2j+2].  Separating-axis test: the two
 * convex sets meet iff their projections overlap on the x axis, the y axis and
 * the segment's normal. */
int orc_segment_meets_cell(int x1, int y1, int x2, int y2, int i, int j) {
    int64_t px = 2 * (int64_t)x1 + 1, py = 2 * (int64_t)y1 + 1;
    int64_t qx = 2 * (int64_t)x2 + 1, qy = 2 * (int64_t)y2 + 1;
    int64_t lo_x = 2 * (int64_t)i, hi_x = lo_x + 2;
    int64_t lo_y = 2 * (int64_t)j, hi_y = lo_y + 2;
    int64_t smin_x = px < qx ? px : qx, smax_x = px < qx ? qx : px;
    int64_t smin_y = py < qy ? py : qy, smax_y = py < qy ? qy : py;
    if (smax_x < lo_x || smin_x > hi_x) return 0;
    if (smax_y < lo_y || smin_y > hi_y) return 0;
    int64_t dx = qx - px, dy = qy - py;
    int64_t cx[4] = {lo_x, hi_x, lo_x, hi_x};
    int64_t cy[4] = {lo_y, lo_y, hi_y, hi_y};
    int pos = 0, neg = 0;
    for (int k = 0; k < 4; k++) {
        int64_t s = dx * (cy[k] - py) - dy * (cx[k] - px);
        if (s > 0) pos++;
        if (s < 0) neg++;
    }
    if (pos == 4 || neg == 4) return 0;
    return 1;
}

/* Brute-force visibility: scan every obstacle cell in the segment's bounding
 * box.  Used to pin the traversal below on small grids. */
int orc_visible_bruteforce(const uint8_t *obst, int W, int H, int x1, int y1, int x2, int y2) {
    int xa = x1 < x2 ? x1 : x2, xb = x1 < x2 ? x2 : x1;
    int ya = y1 < y2 ? y1 : y2, yb = y1 < y2 ? y2 : y1;
    for (int j = ya; j <= yb; j++)
        for (int i = xa; i <= xb; i++)
            if (is_obst(obst, W, H, i, j) && orc_segment_meets_cell(x1, y1, x2, y2, i, j)) return 0;
    return 1;
}

/* Supercover traversal: walk the cells the segment passes through, in order.
 * Between centres the segment crosses the vertical grid lines at parameters
 * (2i+1)/(2|dx|), i = 0..|dx|-1, and the horizontal ones at (2j+1)/(2|dy|).
 * Whichever comes first is the next step; when both coincide the segment goes
 * through a grid corner and touches all four cells around it. */
int orc_visible_dda(const uint8_t *obst, int W, int H, int x1, int y1, int x2, int y2) {
    int dx = x2 - x1, dy = y2 - y1;
    int sx = dx > 0 ? 1 : (dx < 0 ? -1 : 0);
    int sy = dy > 0 ? 1 : (dy < 0 ? -1 : 0);
    int64_t ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
    int x = x1, y = y1;
    int64_t i = 0, j = 0;
    if (is_obst(obst, W, H, x, y)) return 0;
    while (i < ax || j < ay) {
        int step; /* 1 = x, 2 = y, 3 = corner */
        if (i == ax) step = 2;
        else if (j == ay) step = 1;
        else {
            int64_t lhs = (2 * i + 1) * ay, rhs = (2 * j + 1) * ax;
            step = lhs < rhs ? 1 : (lhs > rhs ? 2 : 3);
        }
        if (step == 1) { x += sx; i++; }
        else if (step == 2) { y += sy; j++; }
        else {
            if (is_obst(obst, W, H, x + sx, y)) return 0;
            if (is_obst(obst, W, H, x, y + sy)) return 0;
            x += sx; y += sy; i++; j++;
        }
        if (is_obst(obst, W, H, x, y)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Main component and node numbering (Sec. 3.1, Sec. 3.2).                   */
/* Two free cells that see each other are joined by a 4-connected chain of   */
/* free cells (the supercover of the segment), and 4-adjacent free cells see */
/* each other, so the components of the visibility graph are the            */
/* 4-connected components of the free cells.  The main component is the     */
/* largest; ties go to the one holding the lowest raster index.  Its cells   */
/* are numbered 0..N-1 in row-major raster order.                            */
/* node_of_cell[W*H] receives the id or -1; returns N.                       */
/* ------------------------------------------------------------------------ */
int64_t orc_main_component(const uint8_t *obst, int W, int H, int32_t *node_of_cell) {
    int64_t C = (int64_t)W * H;
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)(C > 0 ? C : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    for (int64_t c = 0; c < C; c++) label[c] = -1;
    int32_t best = -1, next_label = 0;
    int64_t best_size = 0;
    for (int64_t c = 0; c < C; c++) {
        if (obst[c] || label[c] >= 0) continue;
        int32_t L = next_label++;
        int64_t head = 0, tail = 0, size = 0;
        label[c] = L;
        queue[tail++] = c;
        while (head < tail) {
            int64_t cur = queue[head++];
            size++;
            int x = (int)(cur % W), y = (int)(cur / W);
            int nx[4] = {x - 1, x + 1, x, x};
            int ny[4] = {y, y, y - 1, y + 1};
            for (int k = 0; k < 4; k++) {
                if (nx[k] < 0 || ny[k] < 0 || nx[k] >= W || ny[k] >= H) continue;
                int64_t nc = (int64_t)ny[k] * W + nx[k];
                if (obst[nc] || label[nc] >= 0) continue;
                label[nc] = L;
                queue[tail++] = nc;
            }
        }
        if (size > best_size) { best_size = size; best = L; } /* strict: first (lowest raster) wins ties */
    }
    int64_t n = 0;
    for (int64_t c = 0; c < C; c++) node_of_cell[c] = (best >= 0 && label[c] == best) ? (int32_t)n++ : -1;
    free(label);
    free(queue);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Adjacency of the main component, by the supercover traversal.            */
/* cell_of_node[N] (raster cell index of each node) must be given.          */
/* orc_visible_from writes node u's sorted neighbour ids and returns the     */
/* count (out may be NULL to count only).                                   */
/* ------------------------------------------------------------------------ */
int64_t orc_visible_from(const uint8_t *obst, int W, int H, const int64_t *cell_of_node, int64_t n,
                         int64_t u, uint32_t *out) {
    int64_t cnt = 0;
    int xu = (int)(cell_of_node[u] % W), yu = (int)(cell_of_node[u] / W);
    for (int64_t v = 0; v < n; v++) {
        if (v == u) continue;
        int xv = (int)(cell_of_node[v] % W), yv = (int)(cell_of_node[v] / W);
        if (orc_visible_dda(obst, W, H, xu, yu, xv, yv)) {
            if (out) out[cnt] = (uint32_t)v;
            cnt++;
        }
    }
    return cnt;
}

typedef struct {
    const uint8_t *obst; int W, H; const int64_t *cell_of_node; int64_t n;
    const int64_t *nodes; int64_t n_nodes; int64_t *counts; const uint64_t *row_ptr; uint32_t *col;
    int nthreads, tid;
} vis_job;

static void *vis_worker(void *arg) {
    vis_job *J = (vis_job *)arg;
    for (int64_t k = J->tid; k < J->n_nodes; k += J->nthreads) {
        int64_t u = J->nodes ? J->nodes[k] : k;
        if (J->col)
            orc_visible_from(J->obst, J->W, J->H, J->cell_of_node, J->n, u, J->col + J->row_ptr[k]);
        else
            J->counts[k] = orc_visible_from(J->obst, J->W, J->H, J->cell_of_node, J->n, u, NULL);
    }
    return NULL;
}

/* Degrees (col == NULL) or neighbour lists (col != NULL, row_ptr given) for
 * a list of nodes (nodes == NULL: all n nodes), on nthreads threads. */
void orc_visibility_lists(const uint8_t *obst, int W, int H, const int64_t *cell_of_node, int64_t n,
                          const int64_t *nodes, int64_t n_nodes, int64_t *counts,
                          const uint64_t *row_ptr, uint32_t *col, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    pthread_t th[256];
    vis_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; t++) {
        vis_job J = {obst, W, H, cell_of_node, n, nodes, n_nodes, counts, row_ptr, col, nthreads, t};
        jobs[t] = J;
        pthread_create(&th[t], NULL, vis_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Delta-compressed CSR (Sec. 3.2).                                          */
/* ------------------------------------------------------------------------ */

/* Unsigned LEB128: 7-bit groups, least significant first, 0x80 marks that
 * another byte follows.  Returns the number of bytes (out may be NULL). */
int orc_leb128_put(uint64_t value, uint8_t *out) {
    int k = 0;
    do {
        uint8_t b = (uint8_t)(value & 0x7F);
        value >>= 7;
        if (value != 0) b |= 0x80;
        if (out) out[k] = b;
        k++;
    } while (value != 0);
    return k;
}

/* Encode sorted neighbour lists given as plain CSR (row_ptr[n+1], col).  First
 * pass (bytes == NULL) fills offsets[n+1] only; second pass writes bytes.
 * Returns the total byte count. */
uint64_t orc_csr_encode(int64_t n, const uint64_t *row_ptr, const uint32_t *col, uint64_t *offsets,
                        uint8_t *bytes) {
    uint64_t pos = 0;
    for (int64_t v = 0; v < n; v++) {
        offsets[v] = pos;
        uint64_t prev = 0;
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            uint64_t w = col[e];
            uint64_t val = (e == row_ptr[v]) ? w : w - prev; /* first absolute, then delta */
            pos += (uint64_t)orc_leb128_put(val, bytes ? bytes + pos : NULL);
            prev = w;
        }
    }
    offsets[n] = pos;
    return pos;
}

/* The NeighborIter of Sec. 3.2: decode one node's byte range lazily.
 * Returns the number of neighbours written to out (out may be NULL), or -1 if
 * the range is malformed (a varint runs past the end or over 5 bytes, an id is
 * >= n, or the list is not strictly increasing). */
int64_t orc_decode_list(const uint8_t *bytes, uint64_t begin, uint64_t end, int64_t n, uint32_t *out) {
    int64_t cnt = 0;
    uint64_t pos = begin, id = 0;
    while (pos < end) {
        uint64_t val = 0;
        int shift = 0, len = 0;
        for (;;) {
            if (pos >= end || len == 5) return -1;
            uint8_t b = bytes[pos++];
            len++;
            val |= (uint64_t)(b & 0x7F) << shift;
            shift += 7;
            if (!(b & 0x80)) break;
        }
        if (cnt > 0 && val == 0) return -1;
        id = (cnt == 0) ? val : id + val;
        if (id > 0xFFFFFFFFULL || id >= (uint64_t)n) return -1;   /* node ids are 32-bit */
        if (out) out[cnt] = (uint32_t)id;
        cnt++;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* HyperLogLog pieces (Sec. 2.3, Sec. 3.3, Alg. 1).                          */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood 2014; Vigna's splitmix64.c): one state
 * increment by the golden-ratio constant, then the output mix. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int leading_zeros64(uint64_t w) {
    int k = 0;
    for (int b = 63; b >= 0; b--) {
        if ((w >> b) & 1) break;
        k++;
    }
    return k;
}

/* Register index and value for node id v: j = top p bits of the hash, rho =
 * position of the first 1 bit in the remaining 64-p bits (1-based), or 65-p
 * when they are all zero. */
void orc_hll_hash(uint64_t v, uint64_t seed, int p, uint32_t *j_out, uint8_t *rho_out) {
    uint64_t h = orc_splitmix64(v ^ seed);
    uint64_t j = h >> (64 - p);
    uint64_t w = h << p;
    int rho = (w == 0) ? 65 - p : leading_zeros64(w) + 1;
    *j_out = (uint32_t)j;
    *rho_out = (uint8_t)rho;
}

/* Alg. 1 initialisation: zero the counters, then insert each node into its
 * own counter.  regs is N x m, node-major, one byte per register.  reg_bits =
 * 4 is the paper's packed format (Sec. 3.3, "two 4-bit registers per byte"):
 * a register holds at most 15, so rho is clamped to 15 (the paper does not say
 * how larger values are stored; clamping is the reading taken). */
void orc_hll_init_bits(int64_t n, int p, uint64_t seed, int reg_bits, uint8_t *regs) {
    int64_t m = (int64_t)1 << p;
    uint8_t cap = (reg_bits == 4) ? 15 : 255;
    memset(regs, 0, (size_t)(n * m));
    for (int64_t v = 0; v < n; v++) {
        uint32_t j;
        uint8_t rho;
        orc_hll_hash((uint64_t)v, seed, p, &j, &rho);
        if (rho > cap) rho = cap;
        if (rho > regs[v * m + j]) regs[v * m + j] = rho;
    }
}

void orc_hll_init(int64_t n, int p, uint64_t seed, uint8_t *regs) { orc_hll_init_bits(n, p, seed, 8, regs); }

/* HLL alpha_m (Flajolet et al. 2007). */
double orc_hll_alpha(int p) {
    double m = (double)((int64_t)1 << p);
    if (p == 4) return 0.673;
    if (p == 5) return 0.697;
    if (p == 6) return 0.709;
    return 0.7213 / (1.0 + 1.079 / m);
}

/* Correctly rounded (round-half-even) conversion of a 128-bit unsigned
 * integer to double, written out bit by bit. */
double orc_u128_to_double(uint64_t hi, uint64_t lo) {
    u128 x = ((u128)hi << 64) | lo;
    if (x == 0) return 0.0;
    int top = 127;
    while (!((x >> top) & 1)) top--;
    if (top < 53) return (double)(uint64_t)x; /* exact */
    int drop = top - 52;                        /* bits below the 53-bit mantissa */
    u128 mant = x >> drop;
    u128 rem = x - (mant << drop);
    u128 half = (u128)1 << (drop - 1);
    if (rem > half || (rem == half && (mant & 1))) mant += 1;
    return ldexp((double)(uint64_t)mant, drop);
}

/* Estimator of Sec. 2.3 / Sec. 3.3 for one counter of m = 2^p registers.
 *   Z = sum_j 2^{-M[j]}, formed exactly as S = Z * 2^{65-p} (an integer below
 *       2^66) and rounded once to double;
 *   E = alpha_m m^2 / Z;
 *   c = m ln(m / V) if E <= 2.5 m and V > 0 (V = zero registers), else E. */
double orc_hll_estimate(const uint8_t *reg, int p) {
    int64_t m = (int64_t)1 << p;
    int K = 65 - p;
    u128 S = 0;
    int64_t V = 0;
    for (int64_t j = 0; j < m; j++) {
        int M = reg[j];
        if (M == 0) V++;
        S += (u128)1 << (K - M);
    }
    double Z = ldexp(orc_u128_to_double((uint64_t)(S >> 64), (uint64_t)S), -K);
    double alpha_mm = orc_hll_alpha(p) * (double)m * (double)m;
    double E = alpha_mm / Z;
    if (E <= 2.5 * (double)m && V > 0) return (double)m * log((double)m / (double)V);
    return E;
}

/* Eq. sumD for one node and one pass t. */
double orc_accumulate(double sum_d, int t, double c_t, double c_prev) {
    double diff = c_t - c_prev;
    double term = (double)t * diff;
    return sum_d + term;
}

/* ------------------------------------------------------------------------ */
/* One union pass, Eq. hll-union, threaded over nodes (each node is          */
/* independent, so the thread count cannot change the result).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n; int p; const uint64_t *offsets; const uint8_t *bytes;
    const uint8_t *cur; uint8_t *next; const int64_t *nodes; int64_t n_nodes;
    int nthreads, tid; int changed; int bad; uint64_t edges;
} union_job;

static void *union_worker(void *arg) {
    union_job *J = (union_job *)arg;
    int64_t m = (int64_t)1 << J->p;
    uint32_t *nb = NULL;
    int64_t cap = 0;
    for (int64_t k = J->tid; k < J->n_nodes; k += J->nthreads) {
        int64_t v = J->nodes ? J->nodes[k] : k;
        int64_t deg = orc_decode_list(J->bytes, J->offsets[v], J->offsets[v + 1], J->n, NULL);
        if (deg < 0) { J->bad = 1; continue; }
        if (deg > cap) { free(nb); cap = deg; nb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap); }
        orc_decode_list(J->bytes, J->offsets[v], J->offsets[v + 1], J->n, nb);
        uint8_t *dst = J->next + (J->nodes ? k : v) * m;
        const uint8_t *own = J->cur + v * m;
        for (int64_t j = 0; j < m; j++) dst[j] = own[j];              /* next[v] <- cur[v] */
        for (int64_t e = 0; e < deg; e++) {                           /* for w in N(v)     */
            const uint8_t *src = J->cur + (int64_t)nb[e] * m;
            for (int64_t j = 0; j < m; j++)
                if (src[j] > dst[j]) dst[j] = src[j];                 /* register-wise max */
        }
        for (int64_t j = 0; j < m; j++)
            if (dst[j] != own[j]) { J->changed = 1; break; }
        J->edges += (uint64_t)deg;
    }
    free(nb);
    return NULL;
}

/* Union pass over all nodes (nodes == NULL, next is N x m) or over a list of
 * nodes (next is n_nodes x m, row k for nodes[k]).  Returns 1 if any register
 * changed, 0 if none, -1 on a malformed list.  *edges receives the number of
 * neighbour unions performed. */
int orc_union_pass(int64_t n, int p, const uint64_t *offsets, const uint8_t *bytes, const uint8_t *cur,
                   uint8_t *next, const int64_t *nodes, int64_t n_nodes, int nthreads, uint64_t *edges) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    union_job jobs[256];
    if (!nodes) n_nodes = n;
    for (int t = 0; t < nthreads; t++) {
        union_job J = {n, p, offsets, bytes, cur, next, nodes, n_nodes, nthreads, t, 0, 0, 0};
        jobs[t] = J;
        pthread_create(&th[t], NULL, union_worker, &jobs[t]);
    }
    int changed = 0, bad = 0;
    uint64_t e = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        changed |= jobs[t].changed;
        bad |= jobs[t].bad;
        e += jobs[t].edges;
    }
    if (edges) *edges = e;
    return bad ? -1 : changed;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 end to end.                                                    */
/*   d <= 0: no depth limit.  conv_mode 0: stop at the first pass that       */
/*   changes no register; 1: stop when max_v (c_t - c_{t-1}) <= 0.5.         */
/*   comp_size (nullable, else N for every node): exact component sizes N_v. */
/*   Outputs: mean_depth[N] = sum_d / (N_v - 1) (NaN when N_v <= 1),         */
/*   ball[N] = c at the last pass, *iters = passes run.                      */
/*   Optional trace: if trace_regs != NULL it receives (max_trace+1) x N x m  */
/*   registers (index 0 = initial); trace_c likewise (max_trace+1) x N.      */
/* Returns 0, or -1 on a malformed CSR.                                       */
/* ------------------------------------------------------------------------ */
int orc_hyperball_bits(int64_t n, const uint64_t *offsets, const uint8_t *bytes, const uint32_t *comp_size,
                       int p, int d, uint64_t seed, int conv_mode, int reg_bits, int nthreads, double *mean_depth,
                       double *ball, int *iters, uint8_t *trace_regs, double *trace_c, int max_trace) {
    int64_t m = (int64_t)1 << p;
    uint8_t *cur = (uint8_t *)malloc((size_t)(n * m > 0 ? n * m : 1));
    uint8_t *next = (uint8_t *)malloc((size_t)(n * m > 0 ? n * m : 1));
    double *c_prev = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *c_cur = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *sum_d = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int rc = 0, t = 0;

    orc_hll_init_bits(n, p, seed, reg_bits, cur);                    /* Alg. 1 init      */
    for (int64_t v = 0; v < n; v++) c_prev[v] = orc_hll_estimate(cur + v * m, p);  /* c_0 */
    if (trace_regs && max_trace >= 0) memcpy(trace_regs, cur, (size_t)(n * m));
    if (trace_c && max_trace >= 0) memcpy(trace_c, c_prev, sizeof(double) * (size_t)n);

    for (t = 1;; t++) {
        if (n == 0) { t = 0; break; }
        int changed = orc_union_pass(n, p, offsets, bytes, cur, next, NULL, 0, nthreads, NULL);
        if (changed < 0) { rc = -1; break; }
        double max_inc = -INFINITY;
        for (int64_t v = 0; v < n; v++) {
            c_cur[v] = orc_hll_estimate(next + v * m, p);
            sum_d[v] = orc_accumulate(sum_d[v], t, c_cur[v], c_prev[v]);
            double inc = c_cur[v] - c_prev[v];
            if (inc > max_inc) max_inc = inc;
        }
        if (trace_regs && t <= max_trace) memcpy(trace_regs + (int64_t)t * n * m, next, (size_t)(n * m));
        if (trace_c && t <= max_trace) memcpy(trace_c + (int64_t)t * n, c_cur, sizeof(double) * (size_t)n);
        double *tmpc = c_prev; c_prev = c_cur; c_cur = tmpc;
        uint8_t *tmpr = cur; cur = next; next = tmpr;                 /* swap             */
        int stop = (conv_mode == 1) ? (max_inc <= 0.5) : (!changed);
        if (stop || (d > 0 && t >= d)) break;
    }
    if (iters) *iters = t;
    if (rc == 0) {
        for (int64_t v = 0; v < n; v++) {
            double nv = comp_size ? (double)comp_size[v] : (double)n;
            mean_depth[v] = (nv <= 1.0) ? NAN : sum_d[v] / (nv - 1.0);
            ball[v] = c_prev[v];
        }
    }
    free(cur); free(next); free(c_prev); free(c_cur); free(sum_d);
    return rc;
}

int orc_hyperball(int64_t n, const uint64_t *offsets, const uint8_t *bytes, const uint32_t *comp_size,
                  int p, int d, uint64_t seed, int conv_mode, int nthreads, double *mean_depth, double *ball,
                  int *iters, uint8_t *trace_regs, double *trace_c, int max_trace) {
    return orc_hyperball_bits(n, offsets, bytes, comp_size, p, d, seed, conv_mode, 8, nthreads, mean_depth, ball,
                              iters, trace_regs, trace_c, max_trace);
}

/* ------------------------------------------------------------------------ */
/* Exact BFS (ground truth for |B(v,t)| and distance sums).                  */
/* dist[N] receives hop distances from src (-1 unreachable).  Returns the    */
/* eccentricity of src, or -1 on a malformed CSR.                            */
/* ------------------------------------------------------------------------ */
int orc_bfs(int64_t n, const uint64_t *offsets, const uint8_t *bytes, int64_t src, int32_t *dist) {
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *nb = NULL;
    int64_t cap = 0;
    for (int64_t v = 0; v < n; v++) dist[v] = -1;
    int64_t head = 0, tail = 0;
    int ecc = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int64_t v = queue[head++];
        int64_t deg = orc_decode_list(bytes, offsets[v], offsets[v + 1], n, NULL);
        if (deg < 0) { ecc = -1; break; }
        if (deg > cap) { free(nb); cap = deg; nb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap); }
        orc_decode_list(bytes, offsets[v], offsets[v + 1], n, nb);
        for (int64_t e = 0; e < deg; e++) {
            int64_t w = nb[e];
            if (dist[w] >= 0) continue;
            dist[w] = dist[v] + 1;
            if (dist[w] > ecc) ecc = dist[w];
            queue[tail++] = w;
        }
    }
    free(nb);
    free(queue);
    return ecc;
}

/* ------------------------------------------------------------------------ */
/* Closed-form VGA metrics (Sec. 3.3, "Metric derivation").                  */
/* From MD(v), the exact component size k = N_v and the degree:            */
/*   RA    = 2 (MD - 1) / (k - 2)                                            */
/*   D_k   = 2 (k (log2((k + 2) / 3) - 1) + 1) / ((k - 1)(k - 2)), the RA of  */
/*           the root of a diamond-shaped graph of k nodes (Hillier & Hanson */
/*           1984; the paper names RRA but prints no normaliser)            */
/*   HH    = 1 / RRA = D_k / RA                                              */
/*   Tekl  = log2((MD + 2) / 3)                                              */
/*   P     = max(0, 1 - RA)                                                  */
/*   PFM   = MD x deg                                                        */
/* k <= 2 leaves RA undefined: HH and P are NaN.  out is N x 4 (HH, Tekl,   */
/* P, PFM) per node.                                                         */
/* ------------------------------------------------------------------------ */
double orc_dvalue(double k) {
    return 2.0 * (k * (log2((k + 2.0) / 3.0) - 1.0) + 1.0) / ((k - 1.0) * (k - 2.0));
}

void orc_metrics(int64_t n, const double *md, const uint32_t *comp_size, const uint32_t *degree, double *out) {
    for (int64_t v = 0; v < n; v++) {
        double k = comp_size ? (double)comp_size[v] : (double)n;
        double m = md[v];
        double hh = NAN, pv = NAN;
        if (k > 2.0) {
            double ra = 2.0 * (m - 1.0) / (k - 2.0);
            hh = orc_dvalue(k) / ra;
            pv = 1.0 - ra;
            if (pv < 0.0) pv = 0.0;
        }
        out[4 * v + 0] = hh;
        out[4 * v + 1] = log2((m + 2.0) / 3.0);
        out[4 * v + 2] = pv;
        out[4 * v + 3] = m * (double)degree[v];
    }
}

/* ------------------------------------------------------------------------ */
/* Hilbert order (Sec. 3.2, "Optional Hilbert reordering").                  */
/* Index of cell (x, y) along the Hilbert curve filling a 2^k x 2^k square, */
/* by the classic quadrant-by-quadrant construction: at each level from the */
/* coarsest, add the quadrant's offset (0, 1, 2, 3 squares of the level in  */
/* curve order) and rotate/reflect the coordinates into the sub-curve's      */
/* frame.                                                                    */
/* ------------------------------------------------------------------------ */
uint64_t orc_hilbert_index(int k, uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (int64_t s = (int64_t)1 << (k - 1); s > 0; s >>= 1) {
        uint32_t rx = (x & (uint32_t)s) ? 1u : 0u;
        uint32_t ry = (y & (uint32_t)s) ? 1u : 0u;
        d += (uint64_t)s * (uint64_t)s * ((3u * rx) ^ ry);
        if (ry == 0) {                 /* rotate the quadrant */
            if (rx == 1) {
                x = (uint32_t)(s - 1) - (x & (uint32_t)(s - 1)) + (x & ~(uint32_t)(s - 1));
                y = (uint32_t)(s - 1) - (y & (uint32_t)(s - 1)) + (y & ~(uint32_t)(s - 1));
            }
            uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}
