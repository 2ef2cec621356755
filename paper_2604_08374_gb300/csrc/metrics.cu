// metrics.cu -- closed-form VGA metrics from Visual Mean Depth (Sec. 3.3,
// "Metric derivation"): Integration [HH], Integration [Tekl], P-value and
// Point First Moment, one thread per node.
#include "vga_common.cuh"

namespace vga {
namespace {

// RRA normaliser: the relative asymmetry of the root of a diamond-shaped graph
// with k nodes, D_k = 2 (k (log2((k + 2) / 3) - 1) + 1) / ((k - 1)(k - 2)).
__device__ __forceinline__ double dvalue(double k) {
    const double l = log2(__ddiv_rn(__dadd_rn(k, 2.0), 3.0));
    const double num = __dmul_rn(2.0, __dadd_rn(__dmul_rn(k, __dsub_rn(l, 1.0)), 1.0));
    return __ddiv_rn(num, __dmul_rn(__dsub_rn(k, 1.0), __dsub_rn(k, 2.0)));
}

__global__ void metrics_kernel(uint32_t n, const double *__restrict__ md, const uint32_t *__restrict__ comp,
                               const uint32_t *__restrict__ degree, double *__restrict__ out) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double k = comp ? (double)comp[v] : (double)n;
    const double m = md[v];
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    double hh = nan, pv = nan;
    if (k > 2.0) {
        const double ra = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(m, 1.0)), __dsub_rn(k, 2.0));
        hh = __ddiv_rn(dvalue(k), ra);
        pv = __dsub_rn(1.0, ra);
        if (pv < 0.0) pv = 0.0;
    }
    out[4 * v + 0] = hh;
    out[4 * v + 1] = log2(__ddiv_rn(__dadd_rn(m, 2.0), 3.0));
    out[4 * v + 2] = pv;
    out[4 * v + 3] = __dmul_rn(m, (double)degree[v]);
}

}  // namespace
}  // namespace vga

using namespace vga;

extern "C" int vga_metrics(const vga_graph *g, const double *mean_depth_dev, double *out_dev, void *stream_ptr) {
    clear_error();
    if (!g || (g->n && (!mean_depth_dev || !out_dev))) {
        set_error("vga_metrics: null argument");
        return VGA_EINVAL;
    }
    if (g->n == 0) return VGA_OK;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    metrics_kernel<<<(g->n + 255) / 256, 256, 0, stream>>>(g->n, mean_depth_dev, g->d_comp, g->d_degree, out_dev);
    count_launch();
    VGA_CHECK_CUDA(cudaGetLastError());
    return VGA_OK;
}
