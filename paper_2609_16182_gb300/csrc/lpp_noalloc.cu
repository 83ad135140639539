// lpp_noalloc.cu -- row activities of a device-resident LP without any
// device allocation (lpp_row_activity_noalloc in lpp.h).
//
// Some callers cannot allocate device memory at the moment they need row
// activities: a GPU LP solver that reserved its whole memory budget up front
// and treats any further allocation as a failure, or a pipeline whose device
// memory is planned once and must not change while it runs.  For them this
// entry point computes the same quantities as the activity step of
// lpp_presolve using only the arrays the caller passes plus one fixed
// scratch array compiled into the library.
//
// Rows of up to kNaLong entries are reduced by one warp each (no scratch).
// Longer rows are split by fixed 4096-entry windows of the entry array; a
// window meets at most two long rows (one that started before it, one that
// starts inside it), so each window stores at most two partial results in
// the scratch array, and a third kernel adds a long row's partials in window
// order.  Every slot a long row reads is written earlier in the same call, so
// nothing in the scratch array has to start at zero.
#include <algorithm>
#include <mutex>

#include "lpp_engine.h"

namespace {

constexpr int kNaWindow = 4096;           // entries per window
constexpr int kNaLong = 4096;             // longer rows use the windows
constexpr int kNaMaxWindows = 1 << 16;    // => at most 268,435,456 nonzeros
constexpr int kNaThreads = 256;

struct WindowPart {
    double2 act[2];   // (min, max) finite parts for slot 0 / slot 1
    int2 ninf[2];     // infinite-term counts
    int32_t row[2];   // which row each slot belongs to (-1: unused)
    int32_t pad[2];
};

// The scratch of lpp_row_activity_noalloc: 4 MiB per device that loads the
// library, held until the process exits; shared by every call.
static __device__ __align__(256) WindowPart g_na_scratch[kNaMaxWindows];

__device__ __forceinline__ bool na_fin(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ double na_norm(double x, double huge) {
    if (x >= huge) return __longlong_as_double(0x7ff0000000000000LL);
    if (x <= -huge) return __longlong_as_double((long long)0xfff0000000000000ULL);
    return x;
}

struct NaArgs {
    int32_t m;
    int64_t nnz;
    const int32_t *rp, *ci;
    const double *val, *lb, *ub;
    double huge;
    double *amin, *amax;
    int32_t *nmin, *nmax;
};

// accumulate entries [b, e) of a row
__device__ __forceinline__ void na_accumulate(const NaArgs &a, int64_t b, int64_t e, int64_t stride, double &smin,
                                              double &smax, int &cmin, int &cmax) {
    for (int64_t k = b; k < e; k += stride) {
        const double v = a.val[k];
        const int32_t j = a.ci[k];
        const double l = na_norm(a.lb[j], a.huge), u = na_norm(a.ub[j], a.huge);
        const bool neg = __double_as_longlong(v) < 0;
        const double bmin = neg ? u : l, bmax = neg ? l : u;
        if (na_fin(bmin)) smin = fma(v, bmin, smin);
        else cmin++;
        if (na_fin(bmax)) smax = fma(v, bmax, smax);
        else cmax++;
    }
}

// one warp per row of at most kNaLong entries
__global__ void __launch_bounds__(kNaThreads) k_na_short(NaArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kNaThreads / 32);
    for (int64_t i = (int64_t)blockIdx.x * (kNaThreads / 32) + (threadIdx.x >> 5); i < a.m; i += warps) {
        const int64_t b = a.rp[i], e = a.rp[i + 1];
        if (e - b > kNaLong) continue;  // warp-uniform
        double smin = 0.0, smax = 0.0;
        int cmin = 0, cmax = 0;
        na_accumulate(a, b + lane, e, 32, smin, smax, cmin, cmax);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            smin += __shfl_xor_sync(0xffffffffu, smin, o);
            smax += __shfl_xor_sync(0xffffffffu, smax, o);
            cmin += __shfl_xor_sync(0xffffffffu, cmin, o);
            cmax += __shfl_xor_sync(0xffffffffu, cmax, o);
        }
        if (lane == 0) {
            a.amin[i] = smin;
            a.amax[i] = smax;
            a.nmin[i] = cmin;
            a.nmax[i] = cmax;
        }
    }
}

// row containing entry e: the last row whose start is <= e (skips empty rows)
__device__ __forceinline__ int32_t na_row_of(const int32_t *rp, int32_t m, int64_t e) {
    int32_t lo = 0, hi = m;  // rp[lo] <= e < rp[hi] holds for the answer lo
    while (hi - lo > 1) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (rp[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T na_block_sum(T v, T *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kNaThreads / 32; w++) t += s_w[w];
    __syncthreads();
    return t;
}

// one block per window: the partials of the (at most two) long rows it meets
__global__ void __launch_bounds__(kNaThreads) k_na_windows(NaArgs a, WindowPart *scratch) {
    __shared__ double s_d[kNaThreads / 32];
    __shared__ int s_i[kNaThreads / 32];
    const int64_t w0 = (int64_t)blockIdx.x * kNaWindow;
    const int64_t w1 = min(a.nnz, w0 + kNaWindow);
    const int32_t r0 = na_row_of(a.rp, a.m, w0);
    const int32_t r1 = na_row_of(a.rp, a.m, w1 - 1);
    for (int slot = 0; slot < 2; slot++) {
        const int32_t r = slot == 0 ? r0 : r1;
        const int64_t rb = a.rp[r], re = a.rp[r + 1];
        const bool use = re - rb > kNaLong && (slot == 0 || r1 != r0);
        if (!use) {  // block-uniform
            if (threadIdx.x == 0) scratch[blockIdx.x].row[slot] = -1;
            continue;
        }
        const int64_t b = max(rb, w0), e = min(re, w1);
        double smin = 0.0, smax = 0.0;
        int cmin = 0, cmax = 0;
        na_accumulate(a, b + threadIdx.x, e, kNaThreads, smin, smax, cmin, cmax);
        smin = na_block_sum(smin, s_d);
        smax = na_block_sum(smax, s_d);
        cmin = na_block_sum(cmin, s_i);
        cmax = na_block_sum(cmax, s_i);
        if (threadIdx.x == 0) {
            WindowPart &p = scratch[blockIdx.x];
            p.act[slot] = make_double2(smin, smax);
            p.ninf[slot] = make_int2(cmin, cmax);
            p.row[slot] = r;
        }
    }
}

// one thread per long row: its window partials added in window order
__global__ void k_na_long(NaArgs a, const WindowPart *scratch) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.m; i += step) {
        const int64_t rb = a.rp[i], re = a.rp[i + 1];
        if (re - rb <= kNaLong) continue;
        double smin = 0.0, smax = 0.0;
        int cmin = 0, cmax = 0;
        for (int64_t w = rb / kNaWindow; w <= (re - 1) / kNaWindow; w++) {
            const int slot = rb <= w * kNaWindow ? 0 : 1;  // started before the window, or inside it
            const WindowPart &p = scratch[w];
            smin += p.act[slot].x;
            smax += p.act[slot].y;
            cmin += p.ninf[slot].x;
            cmax += p.ninf[slot].y;
        }
        a.amin[i] = smin;
        a.amax[i] = smax;
        a.nmin[i] = cmin;
        a.nmax[i] = cmax;
    }
}

// device address of g_na_scratch, looked up once per device
std::mutex g_na_mu;
void *g_na_ptr[256] = {};

}  // namespace

extern "C" lpp_status lpp_row_activity_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                               const int32_t *col_idx, const double *val, const double *lb,
                                               const double *ub, double huge, double *act_min, double *act_max,
                                               int32_t *ninf_min, int32_t *ninf_max, void *stream) {
    if (m < 0 || n < 0 || nnz < 0 || !(huge > 0))
        return lpp_noalloc_fail(LPP_ERR_INVALID, "lpp_row_activity_noalloc: negative size or huge <= 0");
    if (nnz > (int64_t)kNaMaxWindows * kNaWindow)
        return lpp_noalloc_fail(LPP_ERR_INVALID,
                                "lpp_row_activity_noalloc: nnz exceeds the fixed scratch (at most 268435456)");
    if (m == 0) return LPP_OK;
    if (!row_ptr || !act_min || !act_max || !ninf_min || !ninf_max || (nnz > 0 && (!col_idx || !val || !lb || !ub)))
        return lpp_noalloc_fail(LPP_ERR_INVALID, "lpp_row_activity_noalloc: NULL array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lpp_noalloc_fail(LPP_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return lpp_noalloc_fail(LPP_ERR_CUDA, "device ordinal out of range");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mu);
        if (!g_na_ptr[dev]) {
            // set-up, once per device, with that device current: the array's
            // address, and all three kernels loaded now (with lazy module
            // loading a kernel is otherwise loaded at its first launch, which
            // for the window kernels is the first call with nnz > 4096)
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            cudaFuncAttributes fa;
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_short);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_windows);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_long);
            if (e != cudaSuccess) return lpp_noalloc_fail(LPP_ERR_CUDA, cudaGetErrorString(e));
            g_na_ptr[dev] = p;
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NaArgs a{m, nnz, row_ptr, col_idx, val, lb, ub, huge, act_min, act_max, ninf_min, ninf_max};
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return lpp_noalloc_fail(LPP_ERR_CUDA, cudaGetErrorString(e));
    const int sms_blocks = std::max(1, sms) * 8;
    const int64_t warp_blocks = ((int64_t)m + kNaThreads / 32 - 1) / (kNaThreads / 32);
    k_na_short<<<(unsigned)std::min<int64_t>(warp_blocks, sms_blocks), kNaThreads, 0, s>>>(a);
    if (nnz > kNaLong) {
        const unsigned windows = (unsigned)((nnz + kNaWindow - 1) / kNaWindow);
        k_na_windows<<<windows, kNaThreads, 0, s>>>(a, static_cast<WindowPart *>(scratch));
        const int64_t row_blocks = ((int64_t)m + 255) / 256;
        k_na_long<<<(unsigned)std::min<int64_t>(row_blocks, sms_blocks), 256, 0, s>>>(
            a, static_cast<const WindowPart *>(scratch));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return lpp_noalloc_fail(LPP_ERR_CUDA, cudaGetErrorString(e));
    return LPP_OK;
}
