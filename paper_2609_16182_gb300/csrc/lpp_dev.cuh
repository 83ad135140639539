// lpp_dev.cuh -- device-side types and helpers shared by the library's kernels.
//
// Layout in device memory (one LP, or one arena holding many LPs back to back
// as one block-diagonal LP in batch and serving mode):
//   CSR  ptr int32[m+1], idx int32[nnz], val f64[nnz]          (rows of A)
//   CSC  ptr int32[n+1], idx int32[nnz], val f64[nnz]          (rows of A^T)
//   rows L, U f64[m] (lhs, rhs), rmap int32[m], lp_row int32[m] (arena only)
//   cols lu double2[n] (lb, ub), c f64[n], cmap int32[n], lp_col int32[n]
// rmap / cmap map a current index to its original index.  Matrices and
// vectors are double-buffered: compaction (S7) writes the other buffer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lpp {

constexpr int kBlock = 256;         // threads per block of the segment kernels
constexpr int kLongMin = 4097;      // segments longer than 4096 entries are chunked
constexpr int kChunk = 4096;        // entries per chunk of a long segment
constexpr int kNumClass = 7;        // 0..5: groups of 1<<c lanes per segment, 6: chunked
constexpr int kNone = 0x7fffffff;   // empty slot of an atomicMin index
constexpr int kScanTile = 2048;     // elements per tile of the device-wide scans
constexpr int kFlatTile = 4096;     // entries per tile of the flat compaction scatter
// a segment the flat scatter copies (at most kFlatTile entries) then spans at
// most two tiles, and a chunk of a long segment holds at most one tile start
static_assert(kLongMin - 1 <= kFlatTile && kChunk <= kFlatTile, "flat tile too small");

// Segment class by length: W = 1 << class lanes per segment for class <= 5,
// chunks of kChunk entries for class 6.  A segment's summation order depends
// only on its own length, never on its neighbours in the launch.
__host__ __device__ __forceinline__ int seg_class(int len) {
    if (len <= 4) return 0;
    if (len <= 8) return 1;
    if (len <= 16) return 2;
    if (len <= 32) return 3;
    if (len <= 64) return 4;
    if (len < kLongMin) return 5;
    return 6;
}

// row record kinds (values of lpp.h)
enum : uint8_t {
    RK_KEPT = 0, RK_EMPTY = 1, RK_REDUNDANT = 2, RK_SINGLETON = 3, RK_PARALLEL = 4, RK_SUBST = 5, RK_DOUBLETON = 6,
    RK_DEPENDENT = 7
};
// column kinds (CK_PARALLEL: merged into a parallel leader column, S5c;
// CK_SUBST: a free column singleton eliminated through its row, S5d;
// CK_DOUBLETON: eliminated through a doubleton equation, S5e)
enum : uint8_t { CK_KEPT = 0, CK_FIXED = 1, CK_EMPTY = 2, CK_PARALLEL = 3, CK_SUBST = 4, CK_DOUBLETON = 5 };
// verdict slots per LP, in step order
enum { V_S2_ROW = 0, V_S3_COL = 1, V_S5_ROW = 2, V_S5E_COL = 3, V_S6_COL = 4, V_SLOTS = 5 };

// Global counters of a round (block-aggregated atomics).
struct DevStatus {
    int32_t rows_removed, cols_fixed, bounds_changed, unmatched;
    int32_t participants, sides_tested, err, nnz_eval;  // nnz_eval: nonzeros of the rows S1 evaluated;
                                                         // sides_tested: entry sides S3 tested
    int32_t cls_r[kNumClass];  // class sizes of the rows after compaction
    int32_t cls_c[kNumClass];  // class sizes of the columns after compaction
    int32_t nchunk_r, nchunk_c;
    int32_t m_new, n_new, nnz_new, nnz_new_t;
};

// one chunk of a long segment: entries [begin, end) of segment `seg`, the
// `lidx`-th long segment of its matrix; chunks of a segment are consecutive
struct Chunk {
    int32_t seg, begin, end, lidx;
};

// A segmented matrix (CSR of A, or CSR of A^T) with its schedule.
struct SegMat {
    const int32_t *ptr;
    const int32_t *idx;
    const double *val;
    const int32_t *order;      // segment ids grouped by class, stable within a class
    const Chunk *chunks;       // chunks of the long segments
    const int32_t *lfirst;     // [long + 1] first chunk of each long segment
    int32_t cnt;               // segments
    int32_t nchunks;
    int32_t cls_start[kNumClass + 1];
};

// Everything a round kernel touches (passed by value).
struct Ctx {
    SegMat A;   // CSR of A
    SegMat T;   // CSR of A^T
    int32_t m, n, nlp, round;
    // rows
    double *L, *U;
    const int32_t *rmap, *lp_row;
    // columns
    double2 *lu;
    double *c;                      // written only by S5d (one product per column and round)
    const int32_t *cmap, *lp_col;
    // t_orig: the CSC T is the input's A^T, never compacted, and the columns
    // stay in their input slots (no step that reads columns' entries is on).
    // rinv maps an input row to its current index, cinv an input column to
    // its slot (-1 once either left); clen: entries per column in the
    // current rows.
    const int32_t *rinv, *cinv, *clen;
    int32_t t_orig;
    // rows whose activities must be recomputed this round (1) and the flags
    // being gathered for the next round; columns whose bounds changed
    const uint8_t *rdirty;
    uint8_t *rdnext;
    uint8_t *cchg;
    // row work
    double2 *act;
    int2 *ninf;
    uint8_t *rkind;
    uint8_t *rwork;                 // S5: 1 = take part in this pass
    unsigned long long *hrow;       // S5 key hash
    int32_t *rslot;
    unsigned long long *mL, *mU;    // S5 merged sides (ordered encoding)
    uint8_t *hasf;
    // column work
    unsigned long long *cand_l, *cand_u;  // accepted implied bounds (ordered encoding)
    uint32_t *ctouch;                     // 1 once the column received a candidate this round
    int32_t *tl_list, *tl_cnt;            // columns that received a candidate this round
    int32_t *cl_list, *cl_cnt;            // columns whose bounds changed this round
    int32_t *cl_nnz;                      // their entries
    uint8_t *ckind;
    double *fixv;
    // S5 table
    unsigned long long *tkey, *tlead;
    int32_t tcap;
    int32_t *s5_out, *s5_out_cnt;   // rows the first pass leaves unmatched (list, count)
    // S5c (parallel columns, opt-in): slot per column in the column table
    // (key, columns per key, a member changed) of capacity ctcap; per
    // original column its key, its group's size and its length after its
    // last S5c
    int32_t *cslot;
    unsigned long long *ctkey;
    int32_t *ctcnt, *ctnew;
    int32_t ctcap;
    unsigned long long *pkey;
    int32_t *pcnt, *plen;
    // long segments
    double2 *ch_act;
    int2 *ch_ninf;
    unsigned long long *ch_hash;
    uint8_t *lneed;
    // records, indexed by original (arena) index
    int32_t *rec_rk, *rec_rr, *rec_ra;
    double *rec_rv;
    int32_t *rec_ck, *rec_cr;
    double *rec_cv;
    int32_t *rec_ca, *rec_cp;       // S5c merges: leader (original index), pass
    double *rec_cm;                 // [4 per column] l_k, u_k, l_j, u_j at the merge
    long long *rec_sb;              // S5d substitutions, per original row: start in the store,
    int32_t *rec_sl;                // entries, right-hand side; the store: columns (original
    double *rec_srhs;               // indices) and coefficients, filled through sub_used
    int32_t *rec_scol;
    double *rec_sval;
    unsigned long long *sub_used;
    // per LP
    const int32_t *lp_round0;       // arena round in which each LP joined (NULL: all in round 1)
    int32_t *verdict;               // [nlp][V_SLOTS] smallest original index
    uint8_t *lp_changed;            // [nlp]
    DevStatus *st;
    double feas_tol, bound_tol, max_implied, par_tol;
    int32_t dual;
    int32_t dualfix;                // S6 by locks (opts.dual_fixing)
    int32_t count_work;             // the activity kernels count evaluated nonzeros and tested sides (timing)
    int32_t list_touched;           // S3' runs on the listed columns (not on all of them): list them
    // bound sources (opts.dual_records): per current column the smallest
    // original row whose bound equals this round's accepted candidate
    // (lower, upper; INT32_MAX: none), consumed by S3'; per original column
    // the source row and round of the final lower and upper bound
    int2 *bsrc;
    int4 *rec_bs;
    int32_t dual_rec;
};

// Compaction work (S6, S7) beyond Ctx.
struct CompactCtx {
    int32_t *r_keep, *r_len, *r_pos, *r_off;   // keep flag, new length, new index, new offset
    int32_t *c_keep, *c_len, *c_pos, *c_off;
    double *shift;                             // per row: sum of a_ij * v_j over fixed j
    int32_t *chr_cnt, *chr_off;                // per CSR chunk: kept entries, offset in segment
    double *chr_shift;
    int32_t *cht_cnt, *cht_off;                // per CSC chunk
    double *contrib;                           // per column: c_j * v_j of fixed columns
    double *offset;                            // [nlp] objective constant
    double *offset_part;                       // two-level sum partials
    int32_t *lp_first, *lp_last;               // [nlp] current column range of each LP
    uint8_t *lp_dead;                          // [nlp] a verdict was reached, or retired
    const uint8_t *lp_retired;                 // [nlp] finished LPs leaving the arena (NULL: none)
    int32_t *tile_a, *tile_t;                  // per flat tile: the CSR / CSC segment holding its first entry
    int32_t *r_ch0, *c_ch0;                    // per long row / column: its first chunk
    int32_t *r_new, *c_new;                    // new index, -1 if dropped
    int32_t *c_lock;                           // per column: 1 locked down, 2 locked up (dual fixing)
    // next buffers
    int32_t *rp2, *ci2;
    double *rv2;
    int32_t *cp2, *ri2;
    double *cv2;
    double *L2, *U2;
    int32_t *rmap2, *lp_row2;
    double2 *lu2;
    double *c2;
    int32_t *cmap2, *lp_col2;
    uint8_t *rdirty2;                          // next round's dirty flags
    double2 *act2;                             // carried results of clean rows
    int2 *ninf2;
    unsigned long long *hrow2;
    // CSC kept in the input's numbering and columns kept in place
    // (Ctx::t_orig): the input-to-current maps, updated in place
    int32_t *rinv, *cinv;
};

// ------------------------------------------------------------------ helpers
// The bit pattern of a double through an opaque move: on a plain bitcast the
// compiler turns tests such as "exponent bits all set" or "all but the sign
// bit zero" back into FP64 comparisons, which run on the scarce FP64 pipe.
__device__ __forceinline__ long long dbits(double x) {
    long long r;
    asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
    return r;
}
// finite test and sign test on the bit pattern (integer pipes, not FP64)
__device__ __forceinline__ bool is_fin(double x) {
    return (dbits(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool is_neg(double x) { return dbits(x) < 0; }
__device__ __forceinline__ double pinf() { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ double ninf_() { return __longlong_as_double((long long)0xfff0000000000000ULL); }
// max(1, |x|) with the comparison done on the bit pattern
__device__ __forceinline__ double max1abs(double x) {
    const long long b = dbits(x) & 0x7fffffffffffffffLL;
    return b > 0x3ff0000000000000LL ? __longlong_as_double(b) : 1.0;
}

// Order-preserving map of a double to uint64: x < y <=> enc(x) < enc(y)
// for all non-NaN x, y (used by atomicMin / atomicMax on doubles).
__device__ __forceinline__ unsigned long long enc_dbl(double x) {
    const unsigned long long b = (unsigned long long)dbits(x);
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dec_dbl(unsigned long long e) {
    const unsigned long long b = (e & 0x8000000000000000ULL) ? (e & 0x7fffffffffffffffULL) : ~e;
    return __longlong_as_double((long long)b);
}
constexpr unsigned long long kEncNegInf = 0x000fffffffffffffULL;  // enc(-inf)
constexpr unsigned long long kEncPosInf = 0xfff0000000000000ULL;  // enc(+inf)

__device__ __forceinline__ void atomic_min_dbl(unsigned long long *p, double v) {
    const unsigned long long e = enc_dbl(v);
    if (e < *((volatile unsigned long long *)p)) atomicMin(p, e);
}
__device__ __forceinline__ void atomic_max_dbl(unsigned long long *p, double v) {
    const unsigned long long e = enc_dbl(v);
    if (e > *((volatile unsigned long long *)p)) atomicMax(p, e);
}

// 64-bit mixer: the output function of SplitMix64 (Steele, Lea, Flood 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Key hashes of S5 and S5c: a segment's key hash is the wrapping sum of one
// mixed value per entry (its index and whether its sign differs from the
// first entry's) plus one for the length, so any split of the segment into
// parts sums to the same hash.
__device__ __forceinline__ unsigned long long entry_hash(int32_t j, bool flip) {
    return mix64(((unsigned long long)(uint32_t)j << 1) | (unsigned long long)flip);
}
__device__ __forceinline__ unsigned long long len_hash(int32_t len) {
    return mix64(0xa0761d6478bd642fULL ^ (unsigned long long)(uint32_t)len);
}

// ------------------------------------------------------------- lane groups
// bits [0, W) set
template <int W>
__device__ __forceinline__ unsigned low_bits() {
    if constexpr (W == 32) return 0xffffffffu;
    else return (1u << W) - 1u;
}
// the lanes of this thread's group of W lanes
template <int W>
__device__ __forceinline__ unsigned group_mask() {
    return low_bits<W>() << ((threadIdx.x & 31) & ~(W - 1));
}
// bits of `bal` (a warp ballot) that belong to this thread's group, shifted to 0
template <int W>
__device__ __forceinline__ unsigned group_bits(unsigned bal) {
    return (bal >> ((threadIdx.x & 31) & ~(W - 1))) & low_bits<W>();
}
// xor butterfly: every lane of the group ends with the same bits (a + b == b + a)
template <int W, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
    return v;
}

// block-aggregated counter: one atomic per block
__device__ __forceinline__ void block_add(int32_t v, int32_t *dst) {
    __shared__ int32_t s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc, v);
    __syncthreads();
    if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

// Appends `value` to list[*cnt ...] for each thread with `want`: one shared
// atomic per thread, one global atomic per block.  Every thread of the block
// must call it.  The order within the list is unspecified.
__device__ __forceinline__ void block_append(bool want, int32_t value, int32_t *cnt, int32_t *list) {
    __shared__ int32_t s_n, s_base;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int32_t pos = want ? atomicAdd(&s_n, 1) : 0;
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_n ? atomicAdd(cnt, s_n) : 0;
    __syncthreads();
    if (want) list[s_base + pos] = value;
}

__device__ __forceinline__ int32_t lp_of_row(const Ctx &C, int32_t i) { return C.lp_row ? C.lp_row[i] : 0; }
__device__ __forceinline__ int32_t lp_of_col(const Ctx &C, int32_t j) { return C.lp_col ? C.lp_col[j] : 0; }
// round number of an LP (1 in the arena round in which it joined)
__device__ __forceinline__ int32_t lp_round(const Ctx &C, int32_t lp) {
    return C.lp_round0 ? C.round - C.lp_round0[lp] + 1 : C.round;
}
// LP lp changed this round.  The flag is stored only while it reads 0:
// nearly every row and column of a single-LP arena sets the same byte, and
// repeated stores to one address serialise in L2.
__device__ __forceinline__ void mark_lp_changed(const Ctx &C, int32_t lp) {
    if (!C.lp_changed[lp]) C.lp_changed[lp] = 1;  // a stale 0 only repeats the store
}

// Which class / block-in-class a block of a group launch serves.
struct GroupGrid {
    int32_t blk_start[7];  // first block of classes 0..5, [6] = total blocks
};
__device__ __forceinline__ int grid_class(const GroupGrid &g, int b) {
    int c = 0;
#pragma unroll
    for (int k = 1; k < 6; k++) c += b >= g.blk_start[k];
    return c;
}

}  // namespace lpp
