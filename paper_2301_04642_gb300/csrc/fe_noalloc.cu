// Gershgorin bounds through a path that allocates nothing (fe_k_gershgorin_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the spectral bounds: a host framework whose caching pool owns every byte of
// the GPU, or a latency-critical loop where cudaMalloc / cudaFree (which
// synchronise the whole device) would stall work on other streams.  The
// context-based fe_k_gershgorin needs fe_create and a pooled slot, both of
// which allocate.  This variant takes no context: its per-row scratch lives in
// a fixed file-scope device array, so a call only launches work.
//
// The array holds kNaMaxRows rows (1 MiB + a 256-byte header): larger n is
// rejected with FE_EINVAL.  Every call on a device shares that one array; the
// header (completion counter, NaN/Inf flag) is cleared by a memset on the
// caller's stream at the start of each call, and calls that overlap in time
// (different streams, or host threads without ordering) race on it.
//
// Set-up: the first call on a device, with that device current, looks up
// the array's device address (cudaGetSymbolAddress, which may load this
// module onto the device) and caches it per device; that first call should
// come before any stream capture.
#include <cfloat>
#include <mutex>
#include <string>

#include "../../include/fe_kernels.h"
#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {
namespace {

constexpr int kNaMaxRows = 32768;
constexpr int kNaHeaderDoubles = 32;  // 256 bytes: counter (u32) and flag (i32) at the front
constexpr int kNaRowsPerBlock = 8;    // one warp per row, 256 threads
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_na_scratch[kNaHeaderDoubles + 4 * kNaMaxRows];

std::mutex g_na_mu;
double *g_na_ptr[kNaMaxDevices] = {};

// One launch: each warp writes its row's Gershgorin record (H_ii -/+ r_i,
// H_ii) to the scratch; the block that finishes last (completion counter)
// reduces all rows in a fixed order and writes out4.
__global__ void __launch_bounds__(256) k_gershgorin_oneshot(const double *H, int n, long long ld,
                                                            double *scratch, double *out4) {
    unsigned int *count = reinterpret_cast<unsigned int *>(scratch);
    int *bad = reinterpret_cast<int *>(scratch) + 1;
    double *rows = scratch + kNaHeaderDoubles;  // 4 doubles per row: lo, hi, diag, unused
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * kNaRowsPerBlock + (threadIdx.x >> 5);
    if (row < n) {
        const double *h = H + static_cast<long long>(row) * ld;
        double s = 0.0;
        int nonfinite = 0;
        for (int j = lane; j < n; j += 32) {
            const double v = h[j];
            if (!isfinite(v)) nonfinite = 1;
            s += fabs(v);
        }
        s = warp_sum(s);
        nonfinite = __any_sync(0xffffffffu, nonfinite);
        if (lane == 0) {
            const double d = h[row];
            const double r = s - fabs(d);
            rows[4 * row + 0] = d - r;
            rows[4 * row + 1] = d + r;
            rows[4 * row + 2] = d;
            if (nonfinite) atomicExch(bad, 1);
            __threadfence();
        }
    }
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    __shared__ double s_lo[256], s_hi[256], s_tr[256];
    const int t = threadIdx.x;
    double lo = DBL_MAX, hi = -DBL_MAX, tr = 0.0;
    for (int i = t; i < n; i += blockDim.x) {
        lo = fmin(lo, __ldcg(rows + 4 * i + 0));
        hi = fmax(hi, __ldcg(rows + 4 * i + 1));
        tr += __ldcg(rows + 4 * i + 2);
    }
    s_lo[t] = lo;
    s_hi[t] = hi;
    s_tr[t] = tr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_lo[t] = fmin(s_lo[t], s_lo[t + o]);
            s_hi[t] = fmax(s_hi[t], s_hi[t + o]);
            s_tr[t] += s_tr[t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        out4[0] = s_lo[0];
        out4[1] = s_hi[0];
        out4[2] = s_tr[0];
        out4[3] = atomicAdd(bad, 0) ? 1.0 : 0.0;
    }
}

// Device address of the scratch on the current device (set up on first use).
int scratch_ptr(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error_string(FE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return set_error_string(FE_EINVAL, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess)
            return set_error_string(FE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_na_ptr[dev];
    return FE_OK;
}

}  // namespace
}  // namespace fe

extern "C" int fe_k_gershgorin_noalloc(const double *H, int64_t n, int64_t ld, double *out4,
                                       void *cuda_stream) {
    using namespace fe;
    if (!H || !out4 || n < 1 || ld < n) return set_error_string(FE_EINVAL, "bad arguments");
    if (n > kNaMaxRows)
        return set_error_string(FE_EINVAL, "n = " + std::to_string(n) +
                                               " exceeds the fixed scratch of the no-alloc path (at most " +
                                               std::to_string(kNaMaxRows) + " rows)");
    double *scr = nullptr;
    const int rc = scratch_ptr(&scr);
    if (rc != FE_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(scr, 0, sizeof(double) * kNaHeaderDoubles, s);
    if (e != cudaSuccess) return set_error_string(FE_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int blocks = static_cast<int>((n + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
    k_gershgorin_oneshot<<<blocks, 32 * kNaRowsPerBlock, 0, s>>>(H, static_cast<int>(n), ld, scr, out4);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error_string(FE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return FE_OK;
}
