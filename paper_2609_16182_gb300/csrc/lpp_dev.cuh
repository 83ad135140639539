// lpp_dev.cuh -- device-side types and helpers shared by the library's kernels.
//
// Layout in device memory (one LP, or one arena of many LPs in batch mode):
//   CSR  ptr int32[m+1], idx int32[nnz], val f64[nnz]          (rows of A)
//   CSC  ptr int32[n+1], idx int32[nnz], val f64[nnz]          (rows of A^T)
//   rows L, U f64[m]   (lhs, rhs)      cols lu double2[n] (lb, ub), c f64[n]
//   maps rmap int32[m], cmap int32[n]  (current -> original index)
// Both matrices and all vectors are double-buffered: compaction (S7) writes
// the next buffer and the driver swaps.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lpp {

constexpr int kBlock = 256;         // threads per block of every segment kernel
constexpr int kLongMin = 4097;      // segments longer than 4096 entries are chunked
constexpr int kChunk = 4096;        // entries per chunk of a long segment
constexpr int kNumClass = 7;        // 0..5: groups of 1<<c lanes per segment, 6: chunked
constexpr int kNone = 0x7fffffff;   // "no index" in atomicMin slots

// segment class by length: lanes per segment W = 1 << class for class <= 5.
// The summation order inside a segment depends only on its length, so every
// row gives the same bits whatever else is in the launch (batch == alone).
__host__ __device__ __forceinline__ int seg_class(int len) {
    if (len <= 4) return 0;
    if (len <= 8) return 1;
    if (len <= 16) return 2;
    if (len <= 32) return 3;
    if (len <= 64) return 4;
    if (len < kLongMin) return 5;
    return 6;
}

// row record kinds (the values of lpp.h)
enum : uint8_t { RK_KEPT = 0, RK_EMPTY = 1, RK_REDUNDANT = 2, RK_SINGLETON = 3, RK_PARALLEL = 4 };
// per-row work flags
enum : uint8_t { RF_UNMATCHED = 1, RF_LEADER = 2 };
// column kinds
enum : uint8_t { CK_KEPT = 0, CK_FIXED = 1, CK_EMPTY = 2 };

// Device status word of a round.  Verdict slots hold the smallest current
// index that proved infeasibility / unboundedness in that step (kNone = none).
struct DevStatus {
    int32_t bad_row_s2, bad_col_s3, bad_row_s5, bad_col_s6;
    int32_t verdict;           // nonzero once any verdict slot is set
    int32_t err;               // internal error bits (bounded waits, checks)
    int32_t rows_removed, cols_fixed, bounds_changed, unmatched;
    int32_t m_new, n_new, nnz_new, nnz_new_csc;
    int32_t cls_r[kNumClass];  // class sizes of the rows of the next round
    int32_t cls_c[kNumClass];  // class sizes of the columns of the next round
    int32_t nchunk_r, nchunk_c;
    int32_t participants;      // rows taking part in S5
    int32_t pad;
    double offset_delta;       // objective constant gained this round
};

// one chunk of a long segment: [begin, end) of segment `seg`, which is the
// `lidx`-th long segment; chunks of one segment are consecutive.
struct Chunk {
    int32_t seg, begin, end, lidx;
};

// A segmented matrix (CSR of A, or of A^T) plus its schedule.
struct SegMat {
    const int32_t *ptr;
    const int32_t *idx;
    const double *val;
    const int32_t *order;      // segment ids grouped by class (stable)
    const Chunk *chunks;       // chunks of the long segments
    const int32_t *lfirst;     // [long count + 1] first chunk of each long segment
    int32_t cnt;               // number of segments
    int32_t cls_start[kNumClass + 1];
    int32_t nchunks;
};

// ------------------------------------------------------------------ encodings
// Order-preserving map of a double to uint64 (for atomicMin / atomicMax):
// x < y  <=>  enc(x) < enc(y) for all non-NaN x, y.
__device__ __forceinline__ unsigned long long enc_dbl(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dec_dbl(unsigned long long e) {
    unsigned long long b = (e & 0x8000000000000000ULL) ? (e & 0x7fffffffffffffffULL) : ~e;
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ bool is_fin(double x) { return fabs(x) < __longlong_as_double(0x7ff0000000000000LL); }

__device__ __forceinline__ void atomic_min_dbl(unsigned long long *p, double v) {
    unsigned long long e = enc_dbl(v);
    if (e < *((volatile unsigned long long *)p)) atomicMin(p, e);
}
__device__ __forceinline__ void atomic_max_dbl(unsigned long long *p, double v) {
    unsigned long long e = enc_dbl(v);
    if (e > *((volatile unsigned long long *)p)) atomicMax(p, e);
}

// 64-bit mixer (the finaliser of SplitMix64, Steele et al. 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// normalised coefficient rounded to qbits mantissa bits (round to nearest on
// the bit pattern), the coefficient part of the parallel-row key (Sec. 3.2)
__device__ __forceinline__ unsigned long long quantise(double x, int qbits) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int drop = 52 - qbits;
    if (drop <= 0) return b;
    b += 1ULL << (drop - 1);
    return b & ~((1ULL << drop) - 1ULL);
}

// --------------------------------------------------------------- lane groups
template <int W>
__device__ __forceinline__ unsigned group_mask() {
    if (W == 32) return 0xffffffffu;
    const int lane = threadIdx.x & 31;
    return ((1u << W) - 1u) << (lane & ~(W - 1));
}
template <int W, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
    return v;
}

}  // namespace lpp
