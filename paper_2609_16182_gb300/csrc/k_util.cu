// k_util.cu -- scans, class binning of segments, stable transpose (A -> A^T)
// and the input checks of ingest (S0).
#include <algorithm>
#include <atomic>

#include "lpp_launch.h"

namespace lpp {

namespace {
std::atomic<int64_t> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kScanThreads = 256;
constexpr int kPerThread = kScanTile / kScanThreads;  // 8

struct Pair {
    int32_t a, b;
};
__device__ __forceinline__ Pair operator+(Pair x, Pair y) { return Pair{x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ Pair operator-(Pair x, Pair y) { return Pair{x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ Pair shfl_up(Pair v, int o) {
    return Pair{__shfl_up_sync(0xffffffffu, v.a, o), __shfl_up_sync(0xffffffffu, v.b, o)};
}
__device__ __forceinline__ int32_t shfl_up(int32_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <class T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ int32_t zero_of<int32_t>() { return 0; }
template <> __device__ __forceinline__ Pair zero_of<Pair>() { return Pair{0, 0}; }

// eight consecutive ints from a[k] (zero past cnt): two 16-byte loads when
// all eight are in range and a + k is 16-byte aligned, else one at a time
__device__ __forceinline__ void load8(const int32_t *a, int64_t k, int64_t cnt, int32_t *v) {
    if (k + 8 <= cnt && (reinterpret_cast<uintptr_t>(a + k) & 15u) == 0) {
        const int4 x = *reinterpret_cast<const int4 *>(a + k), y = *reinterpret_cast<const int4 *>(a + k + 4);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = k + q < cnt ? a[k + q] : 0;
    }
}
// eight consecutive ints to a[k] (those before cnt), the same way
__device__ __forceinline__ void store8(int32_t *a, int64_t k, int64_t cnt, const int32_t *v) {
    if (k + 8 <= cnt && (reinterpret_cast<uintptr_t>(a + k) & 15u) == 0) {
        *reinterpret_cast<int4 *>(a + k) = make_int4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<int4 *>(a + k + 4) = make_int4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (k + q < cnt) a[k + q] = v[q];
    }
}

// inputs of a scan: one array, or two arrays scanned together
struct In1 {
    const int32_t *a;
    __device__ int32_t operator()(int64_t k) const { return a[k]; }
    __device__ void get8(int64_t k, int64_t cnt, int32_t *v) const { load8(a, k, cnt, v); }
};
struct In2 {
    const int32_t *a, *b;
    __device__ Pair operator()(int64_t k) const { return Pair{a[k], b[k]}; }
    __device__ void get8(int64_t k, int64_t cnt, Pair *v) const {
        int32_t x[8], y[8];
        load8(a, k, cnt, x);
        load8(b, k, cnt, y);
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = Pair{x[q], y[q]};
    }
};
struct Out1 {
    int32_t *a;
    __device__ void operator()(int64_t k, int32_t v) const { a[k] = v; }
    __device__ void put8(int64_t k, int64_t cnt, const int32_t *v) const { store8(a, k, cnt, v); }
};
struct Out2 {
    int32_t *a, *b;
    __device__ void operator()(int64_t k, Pair v) const {
        a[k] = v.a;
        b[k] = v.b;
    }
    __device__ void put8(int64_t k, int64_t cnt, const Pair *v) const {
        int32_t x[8], y[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            x[q] = v[q].a;
            y[q] = v[q].b;
        }
        store8(a, k, cnt, x);
        store8(b, k, cnt, y);
    }
};

// exclusive scan of the per-thread values of one block; returns the block total
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T &excl, T *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = shfl_up(x, o);
        if (lane >= o) x = x + y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        T acc = zero_of<T>();
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            const T t = s_w[w];
            s_w[w] = acc;
            acc = acc + t;
        }
        s_w[32] = acc;
    }
    __syncthreads();
    excl = s_w[warp] + x - v;
    const T total = s_w[32];
    __syncthreads();
    return total;
}

template <class T, class In>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(In in, int64_t cnt, T *tsum) {
    __shared__ T s_w[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T v = zero_of<T>();
    for (int t = threadIdx.x; t < kScanTile; t += kScanThreads) {
        const int64_t k = base + t;
        if (k < cnt) v = v + in(k);
    }
    T ex;
    const T tot = block_excl_scan(v, ex, s_w);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// one block: exclusive scan of tsum[0..ntiles) in place, tsum[ntiles] = out[cnt] = total
template <class T, class Out>
__global__ void __launch_bounds__(1024) k_scan_top(T *tsum, int32_t ntiles, Out out, int64_t cnt) {
    __shared__ T s_w[33];
    T carry = zero_of<T>();
    for (int32_t b = 0; b < ntiles; b += 1024) {
        const int32_t k = b + threadIdx.x;
        const T v = k < ntiles ? tsum[k] : zero_of<T>();
        T ex;
        const T tot = block_excl_scan(v, ex, s_w);
        if (k < ntiles) tsum[k] = carry + ex;
        carry = carry + tot;
    }
    if (threadIdx.x == 0) {
        tsum[ntiles] = carry;
        out(cnt, carry);
    }
}

template <class T, class In, class Out>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(In in, Out out, int64_t cnt, const T *tsum) {
    __shared__ T s_w[33];
    static_assert(kPerThread == 8, "the scan's thread step is eight values");
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kPerThread;
    T v[kPerThread];
    in.get8(base, cnt, v);
    T s = zero_of<T>();
#pragma unroll
    for (int q = 0; q < kPerThread; q++) s = s + v[q];
    T ex;
    block_excl_scan(s, ex, s_w);
    T run = tsum[blockIdx.x] + ex;
    T o[kPerThread];
#pragma unroll
    for (int q = 0; q < kPerThread; q++) {
        o[q] = run;
        run = run + v[q];
    }
    out.put8(base, cnt, o);
}

// --------------------------------------------------------------- binning
__global__ void __launch_bounds__(kScanThreads) k_bin_hist(const int32_t *ptr, const int32_t *cnt_dev,
                                                           int32_t *hist, int32_t ntiles) {
    __shared__ int32_t s_h[kNumClass];
    const int32_t cnt = *cnt_dev;
    if (threadIdx.x < kNumClass) s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int t = threadIdx.x; t < kScanTile; t += kScanThreads) {
        const int64_t sg = base + t;
        if (sg < cnt) atomicAdd(&s_h[seg_class(ptr[sg + 1] - ptr[sg])], 1);
    }
    __syncthreads();
    if (threadIdx.x < kNumClass) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s_h[threadIdx.x];
}

__global__ void __launch_bounds__(kScanThreads) k_bin_scatter(const int32_t *ptr, const int32_t *cnt_dev,
                                                              const int32_t *off, int32_t ntiles, int32_t *order) {
    __shared__ int32_t s_run[kNumClass];
    const int32_t cnt = *cnt_dev;
    __shared__ int32_t s_w[kScanThreads / 32][kNumClass];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x < kNumClass) s_run[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int r = 0; r < kPerThread; r++) {
        const int64_t sg = base + (int64_t)r * kScanThreads + threadIdx.x;
        const bool valid = sg < cnt;
        const int c = valid ? seg_class(ptr[sg + 1] - ptr[sg]) : kNumClass;
        int rank = 0;
#pragma unroll
        for (int k = 0; k < kNumClass; k++) {
            const unsigned bal = __ballot_sync(0xffffffffu, c == k);
            if (c == k) rank = __popc(bal & lt);
            if (lane == 0) s_w[warp][k] = __popc(bal);
        }
        __syncthreads();
        if (valid) {
            int32_t pre = s_run[c];
            for (int w = 0; w < warp; w++) pre += s_w[w][c];
            order[off[(int64_t)c * ntiles + blockIdx.x] + pre + rank] = (int32_t)sg;
        }
        __syncthreads();
        if (threadIdx.x < kNumClass) {
            int32_t t = 0;
            for (int w = 0; w < kScanThreads / 32; w++) t += s_w[w][threadIdx.x];
            s_run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

// class sizes from the scanned histogram
// one block: exclusive scan in place of the 7 x ntiles class-by-tile counts
// (class-major), the total at a[cnt], and the class sizes
__global__ void __launch_bounds__(1024) k_scan_small_cls(int32_t *a, int32_t cnt, int32_t ntiles, int32_t *cls_out) {
    __shared__ int32_t s_w[33];
    int32_t carry = 0;
    for (int32_t b = 0; b < cnt; b += 1024) {
        const int32_t k = b + threadIdx.x;
        const int32_t v = k < cnt ? a[k] : 0;
        int32_t ex;
        const int32_t tot = block_excl_scan(v, ex, s_w);
        if (k < cnt) a[k] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) a[cnt] = carry;
    __syncthreads();
    if (threadIdx.x < kNumClass)
        cls_out[threadIdx.x] = a[(int64_t)(threadIdx.x + 1) * ntiles] - a[(int64_t)threadIdx.x * ntiles];
}

// one block: the chunks of the long segments (class 6, in schedule order),
// their first chunk (lfirst, with the total at lfirst[long count]) and the count
__global__ void __launch_bounds__(1024) k_chunks(const int32_t *ptr, const int32_t *order, const int32_t *off,
                                                 int32_t ntiles, const int32_t *cls, int32_t cap_long,
                                                 int32_t *lfirst, Chunk *chunks, int32_t *nchunk_out) {
    __shared__ int32_t s_w[33];
    const int32_t nlong = min(cls[6], cap_long);
    const int32_t *lo = order + off[(int64_t)6 * ntiles];
    int32_t carry = 0;
    for (int32_t b = 0; b < nlong; b += 1024) {
        const int32_t t = b + threadIdx.x;
        int32_t sg = 0, pb = 0, pe = 0, v = 0;
        if (t < nlong) {
            sg = lo[t];
            pb = ptr[sg];
            pe = ptr[sg + 1];
            v = (pe - pb + kChunk - 1) / kChunk;
        }
        int32_t ex;
        const int32_t tot = block_excl_scan(v, ex, s_w);
        if (t < nlong) {
            int32_t q = carry + ex;
            lfirst[t] = q;
            for (int32_t k = pb; k < pe; k += kChunk, q++) {
                Chunk ch;
                ch.seg = sg;
                ch.begin = k;
                ch.end = min(pe, k + kChunk);
                ch.lidx = t;
                chunks[q] = ch;
            }
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        lfirst[nlong] = carry;
        *nchunk_out = carry;
    }
}

// ----------------------------------------------------------- input checks
enum : int32_t { ERR_PTR = 1, ERR_COL = 2, ERR_VAL = 4, ERR_ORDER = 8, ERR_VEC = 16 };

__global__ void k_check_ptr(const int32_t *ptr, int32_t m, int64_t nnz, int32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > m) return;
    const int32_t p = ptr[i];
    bool bad = p < 0 || (int64_t)p > nnz;
    if (i == 0) bad |= p != 0;
    if (i == m) bad |= (int64_t)p != nnz;
    if (i < m) bad |= ptr[i + 1] < p;
    if (bad) atomicOr(err, ERR_PTR);
}

// Row of every entry (row_of) and the entry checks, one tile of kRowTile
// entries per block: the rows starting in the tile mark their first entry,
// a block max-scan spreads the marks, then the entries are checked (column
// in range, value finite and nonzero, columns increasing inside a row).
// Searches and marks stay inside [0, m) and the tile even for a malformed
// ptr, which k_check_ptr reports.
constexpr int kRowTile = 4096;
constexpr int kRowPer = kRowTile / kScanThreads;  // 16

// largest r in [0, m - 1] with ptr[r] <= k (0 if none), for non-decreasing ptr
__device__ __forceinline__ int32_t row_search(const int32_t *ptr, int32_t m, int64_t k) {
    int32_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)ptr[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kScanThreads) k_rows_check(const int32_t *ptr, const int32_t *idx, const double *val,
                                                             int32_t m, int32_t n, int64_t nnz, int32_t *row_of,
                                                             int32_t *err) {
    __shared__ int32_t s_row[kRowTile];
    __shared__ int32_t s_wmax[kScanThreads / 32];
    __shared__ int32_t s_r[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * kRowTile;
    const int32_t len = (int32_t)(nnz - k0 < kRowTile ? nnz - k0 : kRowTile);
    for (int x = tid; x < kRowTile; x += kScanThreads) s_row[x] = -1;
    if (tid < 2) s_r[tid] = row_search(ptr, m, tid == 0 ? k0 : k0 + len - 1);
    __syncthreads();
    const int32_t r0 = s_r[0], r1 = s_r[1];
    for (int64_t r = (int64_t)r0 + tid; r <= r1; r += kScanThreads) {
        int64_t x = (int64_t)ptr[r] - k0;
        if (x < 0) x = 0;
        if (x < len) atomicMax(&s_row[x], (int32_t)r);
    }
    __syncthreads();
    {  // inclusive max-scan, 16 consecutive positions per thread
        const int x0 = tid * kRowPer;
        int32_t v[kRowPer], run = -1;
#pragma unroll
        for (int e = 0; e < kRowPer; e++) {
            v[e] = s_row[x0 + e];
            run = v[e] > run ? v[e] : run;
        }
        int32_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o && y > inc) inc = y;
        }
        if (lane == 31) s_wmax[warp] = inc;
        int32_t prev = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) prev = -1;
        __syncthreads();
        for (int w = 0; w < warp; w++) prev = s_wmax[w] > prev ? s_wmax[w] : prev;
        run = prev;
#pragma unroll
        for (int e = 0; e < kRowPer; e++) {
            run = v[e] > run ? v[e] : run;
            s_row[x0 + e] = run < 0 ? r0 : run;
        }
    }
    __syncthreads();
    int32_t e = 0;
    for (int x = tid; x < len; x += kScanThreads) {
        const int64_t k = k0 + x;
        const int32_t r = s_row[x];
        row_of[k] = r;
        const int32_t j = idx[k];
        const double a = val[k];
        if (j < 0 || j >= n) e |= ERR_COL;
        if (!is_fin(a) || a == 0.0) e |= ERR_VAL;
        if (k > 0 && (int64_t)ptr[r] < k && idx[k - 1] >= j) e |= ERR_ORDER;  // k - 1 in the same row
    }
    if (e) atomicOr(err, e);
}

__device__ __forceinline__ double norm_inf(double x, double huge) {
    if (x >= huge) return __longlong_as_double(0x7ff0000000000000LL);
    if (x <= -huge) return __longlong_as_double((long long)0xfff0000000000000ULL);
    return x;
}

__global__ void k_ingest_rows(const double *lhs, const double *rhs, int32_t m, double huge, double *L, double *U,
                              int32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double l = lhs[i], u = rhs[i];
    if (isnan(l) || isnan(u)) atomicOr(err, ERR_VEC);
    const double nl = norm_inf(l, huge), nu = norm_inf(u, huge);
    if ((!is_fin(nl) && !is_neg(nl)) || (!is_fin(nu) && is_neg(nu))) atomicOr(err, ERR_VEC);
    L[i] = nl;
    U[i] = nu;
}

__global__ void k_ingest_cols(const double *lb, const double *ub, const double *c, int32_t n, double huge,
                              double2 *lu, double *cc, int32_t *err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double l = lb[j], u = ub[j], cj = c[j];
    if (isnan(l) || isnan(u) || !is_fin(cj)) atomicOr(err, ERR_VEC);
    const double nl = norm_inf(l, huge), nu = norm_inf(u, huge);
    if ((!is_fin(nl) && !is_neg(nl)) || (!is_fin(nu) && is_neg(nu))) atomicOr(err, ERR_VEC);
    lu[j] = make_double2(nl, nu);
    cc[j] = cj;
}

// ------------------------------------------------------ stable transpose
// LSD radix sort of the entries by column, 8 bits per pass, tiles of
// kRadixTile keys.  Each warp owns a contiguous chunk of 512 keys of its tile
// and ranks them with a running per-warp digit count; the tile is then sorted
// stably in shared memory and written out digit run by digit run (coalesced).
constexpr int kRadixTile = 4096;
constexpr int kRadixWarps = kScanThreads / 32;
constexpr int kRadixChunk = kRadixTile / kRadixWarps;  // 512 keys per warp
constexpr int kRadixSteps = kRadixChunk / 32;          // 16

// lanes of the warp holding the same 8-bit digit d (d = 256: none), from 9
// independent full-warp ballots; every lane of the warp must call it
__device__ __forceinline__ unsigned digit_peers(int d) {
    unsigned m = __ballot_sync(0xffffffffu, d < 256);
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1);
        m &= ((d >> b) & 1) ? bb : ~bb;
    }
    return d < 256 ? m : 0u;
}

__global__ void __launch_bounds__(kScanThreads) k_radix_hist(const uint32_t *keys, int64_t cnt, int shift,
                                                             int32_t *hist, int32_t ntiles) {
    __shared__ int32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int t = threadIdx.x; t < kRadixTile; t += kScanThreads) {
        const int64_t k = base + t;
        if (k < cnt) atomicAdd(&s_h[(keys[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s_h[threadIdx.x];
}

struct RadixOut {
    uint32_t *kout;
    int32_t *vout;  // payload: the entry index
};

// first: the payload is the entry index itself (vin unused)
__global__ void __launch_bounds__(kScanThreads) k_radix_scatter(const uint32_t *kin, const int32_t *vin, bool first,
                                                                int64_t cnt, int shift, const int32_t *off,
                                                                int32_t ntiles, RadixOut o) {
    __shared__ int32_t s_wh[kRadixWarps][256];
    __shared__ int32_t s_dbase[256];
    __shared__ int32_t s_goff[256];
    __shared__ int32_t s_wsum[kRadixWarps];
    __shared__ uint32_t s_k[kRadixTile];
    __shared__ int32_t s_v[kRadixTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = 0; w < kRadixWarps; w++) s_wh[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    int32_t rk[kRadixSteps];
    int dg[kRadixSteps];
#pragma unroll
    for (int i = 0; i < kRadixSteps; i++) {  // all loads first
        const int64_t k = base + warp * kRadixChunk + i * 32 + lane;
        dg[i] = k < cnt ? (int)((kin[k] >> shift) & 255u) : 256;
    }
#pragma unroll
    for (int i = 0; i < kRadixSteps; i++) {
        const int d = dg[i];
        const unsigned peers = digit_peers(d);
        const int run = d < 256 ? s_wh[warp][d] : 0;
        rk[i] = run + __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
        if (d < 256 && lane == __ffs(peers) - 1) s_wh[warp][d] = run + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warps in order, then the tile's digits in order
    const int d0 = threadIdx.x;
    int32_t tot = 0;
    for (int w = 0; w < kRadixWarps; w++) {
        const int32_t c = s_wh[w][d0];
        s_wh[w][d0] = tot;
        tot += c;
    }
    int32_t inc = tot;
#pragma unroll
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o2);
        if (lane >= o2) inc += y;
    }
    if (lane == 31) s_wsum[warp] = inc;
    s_goff[d0] = off[(int64_t)d0 * ntiles + blockIdx.x];
    __syncthreads();
    int32_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += s_wsum[w];
    s_dbase[d0] = wpre + inc - tot;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRadixSteps; i++) {  // the keys again (L1/L2), now to their sorted slots
        const int64_t k = base + warp * kRadixChunk + i * 32 + lane;
        if (k < cnt) {
            const uint32_t key = kin[k];
            const int d = (int)((key >> shift) & 255u);
            const int32_t p = s_dbase[d] + s_wh[warp][d] + rk[i];
            s_k[p] = key;
            s_v[p] = first ? (int32_t)k : vin[k];
        }
    }
    __syncthreads();
    const int32_t ntile = (int32_t)(cnt - base < kRadixTile ? cnt - base : kRadixTile);
    for (int q = threadIdx.x; q < ntile; q += kScanThreads) {
        const uint32_t kk = s_k[q];
        const int d = (int)((kk >> shift) & 255u);
        const int32_t g = s_goff[d] + (q - s_dbase[d]);
        o.kout[g] = kk;
        o.vout[g] = s_v[q];
    }
}

__global__ void k_gather_t(const int32_t *perm, const int32_t *row_of, const double *val, int64_t nnz,
                           int32_t *tidx, double *tval) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int32_t e = perm[p];
    tidx[p] = row_of[e];
    tval[p] = val[e];
}

// A^T row pointers from the sorted column keys: key[p] starts column j's
// run at p for every j in (key[p-1], key[p]]; columns after the last key end at nnz
__global__ void k_colptr_from_keys(const uint32_t *key, int64_t nnz, int32_t n, int32_t *tptr) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int32_t kp = (int32_t)key[p];
    const int32_t kq = p == 0 ? -1 : (int32_t)key[p - 1];
    for (int32_t j = kq + 1; j <= kp; j++) tptr[j] = (int32_t)p;
    if (p == nnz - 1)
        for (int32_t j = kp + 1; j <= n; j++) tptr[j] = (int32_t)nnz;
}

// segment lengths from a pointer array
__global__ void k_ptr_diff(const int32_t *ptr, int32_t cnt, int32_t *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = ptr[i + 1] - ptr[i];
}

__global__ void k_iota(int32_t *a, int32_t cnt, int32_t base) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < cnt) a[k] = base + (int32_t)k;
}

__global__ void k_fill_u64(unsigned long long *a, int64_t cnt, unsigned long long v) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < cnt) a[k] = v;
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)std::max<int64_t>(1, (cnt + threads - 1) / threads);
}

}  // namespace

// ================================================================= host side
// int32 elements of scan temporary: room for pair tile sums
size_t scan_tmp_elems(int64_t cnt) { return 2 * ((size_t)((cnt + kScanTile - 1) / kScanTile) + 1); }

void scan_excl(const int32_t *in, int32_t *out, int64_t cnt, int32_t *tmp, cudaStream_t s) {
    const int32_t ntiles = (int32_t)((cnt + kScanTile - 1) / kScanTile);
    if (ntiles > 0) (k_scan_reduce<int32_t><<<ntiles, kScanThreads, 0, s>>>(In1{in}, cnt, tmp), note_launch());
    (k_scan_top<int32_t><<<1, 1024, 0, s>>>(tmp, ntiles, Out1{out}, cnt), note_launch());
    if (ntiles > 0) (k_scan_down<int32_t><<<ntiles, kScanThreads, 0, s>>>(In1{in}, Out1{out}, cnt, tmp), note_launch());
}

void scan_excl2(const int32_t *a, const int32_t *b, int32_t *oa, int32_t *ob, int64_t cnt, int32_t *tmp,
                cudaStream_t s) {
    const int32_t ntiles = (int32_t)((cnt + kScanTile - 1) / kScanTile);
    Pair *t = reinterpret_cast<Pair *>(tmp);
    if (ntiles > 0) (k_scan_reduce<Pair><<<ntiles, kScanThreads, 0, s>>>(In2{a, b}, cnt, t), note_launch());
    (k_scan_top<Pair><<<1, 1024, 0, s>>>(t, ntiles, Out2{oa, ob}, cnt), note_launch());
    if (ntiles > 0) (k_scan_down<Pair><<<ntiles, kScanThreads, 0, s>>>(In2{a, b}, Out2{oa, ob}, cnt, t), note_launch());
}

size_t sched_tile_hist_elems(int64_t cnt) {
    return (size_t)kNumClass * (size_t)std::max<int64_t>(1, (cnt + kScanTile - 1) / kScanTile) + 1;
}

int32_t sched_cap_long(int64_t nnz) { return (int32_t)std::max<int64_t>(1, nnz / kLongMin); }

void build_schedule(const int32_t *ptr, const int32_t *cnt_dev, int32_t cnt_max, int64_t nnz_max,
                    const SchedBufs &b, int32_t *cls_out, int32_t *nchunk_out, cudaStream_t s) {
    // tiles cover cnt_max segments; tiles past the actual count hold zeros
    const int32_t ntiles = std::max<int32_t>(1, (int32_t)((cnt_max + kScanTile - 1) / kScanTile));
    (k_bin_hist<<<ntiles, kScanThreads, 0, s>>>(ptr, cnt_dev, b.tile_hist, ntiles), note_launch());
    (k_scan_small_cls<<<1, 1024, 0, s>>>(b.tile_hist, kNumClass * ntiles, ntiles, cls_out), note_launch());
    (k_bin_scatter<<<ntiles, kScanThreads, 0, s>>>(ptr, cnt_dev, b.tile_hist, ntiles, b.order), note_launch());
    // chunks of the long segments: at most nnz / kLongMin of them
    const int32_t cap_long = sched_cap_long(nnz_max);
    (k_chunks<<<1, 1024, 0, s>>>(ptr, b.order, b.tile_hist, ntiles, cls_out, cap_long, b.lfirst, b.chunks,
                                 nchunk_out), note_launch());
}

void segmat_from_counts(SegMat &M, const int32_t cls[kNumClass], int32_t nchunks) {
    M.cls_start[0] = 0;
    for (int c = 0; c < kNumClass; c++) M.cls_start[c + 1] = M.cls_start[c] + cls[c];
    M.nchunks = nchunks;
}

GroupGrid group_grid(const SegMat &M) {
    GroupGrid g;
    int32_t acc = 0;
    for (int c = 0; c < 6; c++) {
        g.blk_start[c] = acc;
        const int32_t per = kBlock >> c;
        const int32_t cnt = M.cls_start[c + 1] - M.cls_start[c];
        acc += (cnt + per - 1) / per;
    }
    g.blk_start[6] = acc;
    return g;
}

void check_csr(const int32_t *ptr, const int32_t *idx, const double *val, int32_t m, int32_t n, int64_t nnz,
               int32_t *row_of, int32_t *tmp, int32_t *err, cudaStream_t s) {
    (void)tmp;
    (k_check_ptr<<<blocks_for((int64_t)m + 1, 256), 256, 0, s>>>(ptr, m, nnz, err), note_launch());
    // row_of[0] is unused (callers read row_of + 1)
    if (nnz > 0 && m > 0)
        (k_rows_check<<<(unsigned)((nnz + kRowTile - 1) / kRowTile), kScanThreads, 0, s>>>(ptr, idx, val, m, n, nnz,
                                                                                           row_of + 1, err),
         note_launch());
}

void ingest_vectors(const double *lhs, const double *rhs, const double *lb, const double *ub, const double *c,
                    int32_t m, int32_t n, double huge, double *L, double *U, double2 *lu, double *cc, int32_t *err,
                    cudaStream_t s) {
    if (m > 0) (k_ingest_rows<<<blocks_for(m, 256), 256, 0, s>>>(lhs, rhs, m, huge, L, U, err), note_launch());
    if (n > 0) (k_ingest_cols<<<blocks_for(n, 256), 256, 0, s>>>(lb, ub, c, n, huge, lu, cc, err), note_launch());
}

size_t transpose_hist_elems(int64_t nnz) { return (size_t)256 * (size_t)((nnz + kRadixTile - 1) / kRadixTile) + 1; }

void transpose(const int32_t *ptr, const int32_t *idx, const double *val, const int32_t *row_of, int32_t m,
               int32_t n, int64_t nnz, const TransposeBufs &b, int32_t *tptr, int32_t *tidx, double *tval,
               cudaStream_t s) {
    (void)ptr;
    (void)m;
    if (nnz == 0) {
        cudaMemsetAsync(tptr, 0, sizeof(int32_t) * (size_t)(n + 1), s);
        return;
    }
    // stable LSD radix sort of the entries by column (entries come row by row)
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) bits++;
    const int passes = bits > 0 ? (bits + 7) / 8 : 1;
    const int32_t ntiles = (int32_t)((nnz + kRadixTile - 1) / kRadixTile);
    const uint32_t *kin = reinterpret_cast<const uint32_t *>(idx);
    const int32_t *vin = nullptr;
    uint32_t *kbuf[2] = {b.k0, b.k1};
    int32_t *vbuf[2] = {b.v0, b.v1};
    for (int p = 0; p < passes; p++) {
        (k_radix_hist<<<ntiles, kScanThreads, 0, s>>>(kin, nnz, 8 * p, b.hist, ntiles), note_launch());
        scan_excl(b.hist, b.hist, (int64_t)256 * ntiles, b.tmp, s);
        RadixOut o{kbuf[p & 1], vbuf[p & 1]};
        (k_radix_scatter<<<ntiles, kScanThreads, 0, s>>>(kin, vin, p == 0, nnz, 8 * p, b.hist, ntiles, o),
         note_launch());
        kin = kbuf[p & 1];
        vin = vbuf[p & 1];
    }
    (k_gather_t<<<blocks_for(nnz, 256), 256, 0, s>>>(vin, row_of, val, nnz, tidx, tval), note_launch());
    (k_colptr_from_keys<<<blocks_for(nnz, 256), 256, 0, s>>>(kin, nnz, n, tptr), note_launch());
}

void sort_pairs(const uint32_t *keys, const int32_t *vals, int64_t cnt, int bits, const TransposeBufs &b,
                const uint32_t **kout, const int32_t **vout, cudaStream_t s) {
    const uint32_t *kin = keys;
    const int32_t *vin = vals;
    if (cnt > 0) {
        const int passes = bits > 8 ? (bits + 7) / 8 : 1;
        const int32_t ntiles = (int32_t)((cnt + kRadixTile - 1) / kRadixTile);
        uint32_t *kbuf[2] = {b.k0, b.k1};
        int32_t *vbuf[2] = {b.v0, b.v1};
        for (int p = 0; p < passes; p++) {
            (k_radix_hist<<<ntiles, kScanThreads, 0, s>>>(kin, cnt, 8 * p, b.hist, ntiles), note_launch());
            scan_excl(b.hist, b.hist, (int64_t)256 * ntiles, b.tmp, s);
            RadixOut o{kbuf[p & 1], vbuf[p & 1]};
            (k_radix_scatter<<<ntiles, kScanThreads, 0, s>>>(kin, vin, false, cnt, 8 * p, b.hist, ntiles, o),
             note_launch());
            kin = kbuf[p & 1];
            vin = vbuf[p & 1];
        }
    }
    *kout = kin;
    *vout = vin;
}

void ptr_diff(const int32_t *ptr, int32_t cnt, int32_t *out, cudaStream_t s) {
    if (cnt > 0) (k_ptr_diff<<<blocks_for(cnt, 256), 256, 0, s>>>(ptr, cnt, out), note_launch());
}

void iota(int32_t *a, int32_t cnt, int32_t base, cudaStream_t s) {
    if (cnt > 0) (k_iota<<<blocks_for(cnt, 256), 256, 0, s>>>(a, cnt, base), note_launch());
}

void fill_u64(unsigned long long *a, int64_t cnt, unsigned long long v, cudaStream_t s) {
    if (cnt > 0) (k_fill_u64<<<blocks_for(cnt, 256), 256, 0, s>>>(a, cnt, v), note_launch());
}

}  // namespace lpp

namespace lpp {
namespace {
__global__ void k_fill_i32(int32_t *a, int64_t cnt, int32_t v) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < cnt) a[k] = v;
}
__global__ void k_split_lu(const double2 *lu, int32_t n, double *lb, double *ub) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double2 b = lu[j];
    lb[j] = b.x;
    ub[j] = b.y;
}
}  // namespace
void fill_i32(int32_t *a, int64_t cnt, int32_t v, cudaStream_t s) {
    if (cnt > 0) (k_fill_i32<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(a, cnt, v), note_launch());
}
void split_lu(const double2 *lu, int32_t n, double *lb, double *ub, cudaStream_t s) {
    if (n > 0) (k_split_lu<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lu, n, lb, ub), note_launch());
}
}  // namespace lpp
