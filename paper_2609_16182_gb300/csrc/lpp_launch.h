// lpp_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "lpp_dev.cuh"

namespace lpp {

// number of kernels the library has launched in this process (all threads)
void note_launch();
int64_t launch_count();

// ----------------------------------------------------------------- k_util.cu
// Exclusive scan of in[0..cnt) into out[0..cnt], out[cnt] = total.  `tmp`
// must hold scan_tmp_elems(cnt) int32 values.  in == out is allowed.
size_t scan_tmp_elems(int64_t cnt);
void scan_excl(const int32_t *in, int32_t *out, int64_t cnt, int32_t *tmp, cudaStream_t s);
// two exclusive scans in one pass (oa[cnt], ob[cnt] = totals)
void scan_excl2(const int32_t *a, const int32_t *b, int32_t *oa, int32_t *ob, int64_t cnt, int32_t *tmp,
                cudaStream_t s);

// Schedule (class lists + chunks) of a segmented matrix with ptr[cnt+1].
struct SchedBufs {
    int32_t *order;     // [cap_seg]
    Chunk *chunks;      // [cap_chunk]
    int32_t *lfirst;    // [cap_long + 1]
    int32_t *tile_hist; // [7 * tiles + 1]
    int32_t *tmp;       // scan temporary
    int32_t *nch;       // [cap_long + 1]
};
size_t sched_tile_hist_elems(int64_t cnt);
// most long segments a matrix with nnz entries can have (sizes lfirst, nch)
int32_t sched_cap_long(int64_t nnz);
// Builds the schedule and writes the class sizes to cls_out[7] and the chunk
// count to *nchunk_out (device addresses inside DevStatus).  Chunks need at
// most nnz / kChunk + cap_long entries.
void build_schedule(const int32_t *ptr, const int32_t *cnt_dev, int32_t cnt_max, int64_t nnz_max,
                    const SchedBufs &b, int32_t *cls_out, int32_t *nchunk_out, cudaStream_t s);
// Fill the host-side part of a SegMat from class sizes read back.
void segmat_from_counts(SegMat &M, const int32_t cls[kNumClass], int32_t nchunks);
GroupGrid group_grid(const SegMat &M);

// Input checks: returns error bits in *err (device).  row_of[nnz] is filled.
void check_csr(const int32_t *ptr, const int32_t *idx, const double *val, int32_t m, int32_t n, int64_t nnz,
               int32_t *row_of, int32_t *tmp, int32_t *err, cudaStream_t s);
// Vectors: normalise |v| >= huge to +-inf, check NaN / wrong-signed infinity,
// interleave (lb, ub) into lu.
void ingest_vectors(const double *lhs, const double *rhs, const double *lb, const double *ub, const double *c,
                    int32_t m, int32_t n, double huge, double *L, double *U, double2 *lu, double *cc, int32_t *err,
                    cudaStream_t s);
// A^T in CSR form (stable: rows increasing inside each column).
struct TransposeBufs {
    uint32_t *k0, *k1;  // keys [nnz]
    int32_t *v0, *v1;   // values [nnz]
    int32_t *hist;      // [transpose_hist_elems(nnz)]
    int32_t *tmp;       // scan temporary
};
size_t transpose_hist_elems(int64_t nnz);
void transpose(const int32_t *ptr, const int32_t *idx, const double *val, const int32_t *row_of, int32_t m,
               int32_t n, int64_t nnz, const TransposeBufs &b, int32_t *tptr, int32_t *tidx, double *tval,
               cudaStream_t s);
// Stable LSD radix sort of cnt (key, value) pairs by the low `bits` bits of
// the keys (8 bits per pass).  keys / vals are not written; the sorted pairs
// end in b.k0/b.v0 or b.k1/b.v1, returned in *kout / *vout (the inputs
// themselves when cnt == 0).  b.hist needs transpose_hist_elems(cnt) entries.
void sort_pairs(const uint32_t *keys, const int32_t *vals, int64_t cnt, int bits, const TransposeBufs &b,
                const uint32_t **kout, const int32_t **vout, cudaStream_t s);
void iota(int32_t *a, int32_t cnt, int32_t base, cudaStream_t s);
void ptr_diff(const int32_t *ptr, int32_t cnt, int32_t *out, cudaStream_t s);  // out[i] = ptr[i+1] - ptr[i]
void fill_u64(unsigned long long *a, int64_t cnt, unsigned long long v, cudaStream_t s);
void fill_i32(int32_t *a, int64_t cnt, int32_t v, cudaStream_t s);
void split_lu(const double2 *lu, int32_t n, double *lb, double *ub, cudaStream_t s);

// ---------------------------------------------------------------- k_round.cu
// S1-S3: the rows of classes 0-5 (launch_prop_short) and the chunked long
// rows (launch_prop_long) touch disjoint rows and meet only in atomics, so
// they may run on two streams at once
void launch_prop_short(const Ctx &C, cudaStream_t s);
void launch_prop_long(const Ctx &C, cudaStream_t s);
bool prop_has_long(const Ctx &C);
// S3 bound sources (opts.dual_records), between S3 and S3'
void launch_bound_src(const Ctx &C, cudaStream_t s);
// rows list[0 .. cnt) (current indices) become dependent rows (kind and records, round C.round)
void launch_mark_dependent(const Ctx &C, const int32_t *list, int32_t cnt, cudaStream_t s);
void launch_colfin(const Ctx &C, bool full, cudaStream_t s);  // full: every column, else the touched list
void launch_mark_dirty(const Ctx &C, int64_t nnz, cudaStream_t s);
void launch_s5_pass(const Ctx &C, cudaStream_t s);
// one later S5 pass over list[0 .. *cnt), *cnt <= max_rows; unmatched rows are appended to out
void launch_s5_tail(const Ctx &C, const int32_t *list, const int32_t *cnt, int32_t *out, int32_t *out_cnt,
                    int32_t max_rows, cudaStream_t s);
// all remaining later S5 passes of a short list in one block (passes p0 ..
// max_iter - 1; rows left after the last one in cnt[max_iter])
void launch_s5_tail_block(const Ctx &C, int32_t *l0, int32_t *l1, int32_t *cnt, int32_t p0, int32_t max_iter,
                          cudaStream_t s);
constexpr int32_t kTailBlockRows = 4096;  // longest list the one-block form takes
// all remaining later S5 passes of a longer list in one cooperative launch
// with grid barriers (bar: two zeroed words kept by the caller); false if
// the launch is not possible
bool launch_s5_tail_grid(const Ctx &C, int32_t *l0, int32_t *l1, int32_t *cnt, int32_t p0, int32_t max_iter,
                         int32_t rows, unsigned *bar, cudaStream_t s);
void launch_s5_leader(const Ctx &C, cudaStream_t s);

// --------------------------------------------------------------- k_parcols.cu
// S5c keys: the key hash of every column S4 left unfixed goes into the
// column table (C.ctcap slots, empty before), which counts the columns per key
void launch_s5c_keys(const Ctx &C, cudaStream_t s);
// the columns of the groups that changed since their last S5c (a key or the
// size) and have two or more columns, in column order: slot[p], col[p] for
// p < pos[n] (flags, pos: n + 1 entries of scratch)
void launch_s5c_members(const Ctx &C, int32_t *flags, int32_t *pos, int32_t *scan_tmp, uint32_t *slot, int32_t *col,
                        cudaStream_t s);
// bytes per grouped column of the launch_s5c_groups scratch `mem`
size_t s5c_mem_bytes();
// all leader passes of every group: F members sorted by slot (column order
// within a slot), one warp per group of at most 256 columns, larger groups
// listed in glist and run by thread blocks.  ctr[0]: groups left unresolved
// at the pass cap, ctr[1]: large groups (both zero before).
void launch_s5c_groups(const Ctx &C, const uint32_t *slot, const int32_t *col, int32_t F, void *mem, uint8_t *alive,
                       int2 *glist, int32_t *ctr, int32_t max_iter, cudaStream_t s);

// --------------------------------------------------------------- k_colsing.cu
// S5d on the current round: candidates (rcand per row, kNone before), the
// eligibility test (relig per row, 0 before; rows of 65 to 4096 entries
// listed in tasks / *ntask, 0 before; longer rows by chunks, their candidate's
// coefficient in cs_a per row), the first bidding row per column (cmin,
// kNone before), then the substitutions
void launch_s5d(const Ctx &C, int32_t *rcand, uint8_t *relig, int32_t *cmin, int32_t *tasks, int32_t *ntask,
                double *cs_a, cudaStream_t s);

// ------------------------------------------------------------- k_doubleton.cu
// S5e work: per row the candidate's eliminated column (dk, -1 if none), the
// smallest candidate claiming the row (rmin, kNone before), selected (dsel),
// for a selected row x_j, f, g (dj, df, dg); per changed row x_j, x_k and
// x_j's coefficient change (dmj, -1 if unchanged, dmk, dmd), the positions
// of x_k and of x_j (dpk, dpj), flags (dfl: 1 x_j present, 2 cancelled)
// and x_j's new coefficient (dnv); per column the smallest claiming
// candidate (cmin, kNone before); the columns x_j of the applied rows
// (jlist); cnt[0] applied doubletons, cnt[1] jlist entries (0 before)
struct S5eBufs {
    int32_t *dk, *rmin, *cmin, *dj, *dmj, *dmk, *dpk, *dpj, *jlist, *cnt;
    uint8_t *dsel, *dfl;
    double *df, *dg, *dmd, *dnv;
};
// candidates, claims, selection and the applied doubletons (bounds, costs,
// sides, records, the changed rows' notes)
void launch_s5e(const Ctx &C, const S5eBufs &D, cudaStream_t s);
// the rewritten row lengths into rlen[0 .. m)
void launch_s5e_rowlen(const Ctx &C, const S5eBufs &D, int32_t *rlen, cudaStream_t s);
// the rewritten CSR (rp2: the scanned lengths) and the row of each of its entries
void launch_s5e_scatter(const Ctx &C, const S5eBufs &D, const int32_t *rp2, int32_t *ci2, double *rv2,
                        int32_t *row_of, int64_t nnz, cudaStream_t s);
// on the rewritten matrices: the rows of the cnt columns in jlist are dirty
void launch_s5e_mark(const Ctx &C, const S5eBufs &D, int32_t cnt, cudaStream_t s);

// ---------------------------------------------------------------- k_batch.cu
// The persistent batch kernel: one thread block per LP at a time, every round
// of the LP on the device (LPs whose rows and columns all have at most 4096
// entries; options without parallel_cols, col_singletons and doubletons).
struct FusedLP {
    int32_t row_off, col_off, nnz_off;  // the LP's ranges in the arena
    int32_t m, n, nnz;
    int32_t tab_off, tcap;              // its S5 table: tcap slots (a power of two >= 2 m) from tab_off
};

// per LP result
struct FusedOut {
    int32_t status, where, index, round, rounds;
    int32_t m, n, nnz;  // reduced sizes
    int32_t act_m;      // rows at the start of the last round
    int32_t pad;
    long long s5_left;  // rows unmatched when the S5 passes stopped at the cap, over all rounds
};

struct FusedArgs {
    Ctx base;         // arena arrays shared by all LPs (row / column work, records, options)
    CompactCtx K;     // arena compaction work
    int32_t *frp[2], *ftp[2];  // CSR / CSC pointers, LP k's at row_off + k / col_off + k (m + 1, n + 1 entries)
    int32_t *ci[2], *ti[2];
    double *rv[2], *tv[2], *L[2], *U[2], *c[2];
    double2 *lu[2];
    int32_t *rmap[2], *cmap[2];
    double2 *act[2];           // row results, carried over for rows not re-evaluated
    int2 *ninf[2];
    unsigned long long *hrow[2];
    uint8_t *rdirty[2];        // rows to evaluate this round (buffer 0: every row, round 1)
    const int32_t *rp0, *tp0;  // pointers of the ingested arena (one entry per row / column + 1)
    int32_t *order;            // rows by length class
    int32_t *list[2];          // S5 lists of unmatched rows
    unsigned long long *tkey, *tlead;
    DevStatus *st;             // per LP
    int32_t *cnt;              // per LP: touched columns, changed columns, their entries
    uint8_t *dead;             // per LP
    const FusedLP *lps;
    const int32_t *queue;      // LP order
    int32_t *next;             // queue head
    int32_t count, max_rounds, par_max_iter;
    FusedOut *out;
    int32_t *rstat;            // per LP and round: nonzeros, rows removed, columns fixed, bounds changed
    // outputs (the LP's ranges; ptr arrays at row_off + k / col_off + k)
    int32_t *o_rp, *o_ci, *o_tp, *o_ti, *o_rmap, *o_cmap, *o_fcmap, *o_armap;
    double *o_rv, *o_tv, *o_L, *o_U, *o_c, *o_lb, *o_ub;
    double2 *o_lu, *o_act;
    int2 *o_ninf;
};

// dynamic shared memory and resident blocks per SM of a launch with `threads`
// (128, 256 or 512) threads per block
size_t batch_fused_smem(int threads);
int batch_fused_blocks_per_sm(int threads);
void launch_batch_fused(const FusedArgs &F, int threads, int blocks, cudaStream_t s);

// -------------------------------------------------------------- k_compact.cu
// a second stream with its fork and join events (work on it starts after
// the fork recorded on the main stream, which waits for the join)
struct SideStream {
    cudaStream_t s;
    cudaEvent_t fork, join;
};
void launch_compact_counts(const Ctx &C, const CompactCtx &K, cudaStream_t s, const SideStream *side = nullptr);
void launch_compact_scatter(const Ctx &C, const CompactCtx &K, int32_t nnz, cudaStream_t s);
// the result's CSC from the input CSC when it was not compacted (Ctx::t_orig):
// counts and keep flags, then (after the caller's column scan) the scatter
void launch_rows_left(const int32_t *rinv, int32_t m, uint8_t *rk, cudaStream_t s);
// columns kept in place (Ctx::t_orig): their keep flags, then (after the
// caller's scan of them into K.c_pos) their vectors to K.lu2 / c2 / cmap2 /
// lp_col2, cinv to final indices and the CSR's column indices renumbered
void launch_cols_alive(const int32_t *cinv, int32_t n, int32_t *keep, cudaStream_t s);
void launch_cols_final(const Ctx &C, const CompactCtx &K, int32_t n, int32_t *cinv, int32_t *idx, int64_t nnz,
                       cudaStream_t s);
void launch_csc_from_input_counts(const Ctx &C, const CompactCtx &K, cudaStream_t s);
void launch_csc_from_input_scatter(const Ctx &C, const CompactCtx &K, int64_t nnz, int32_t *ptr, int32_t *idx,
                                   double *val, cudaStream_t s);
void launch_offset(const Ctx &C, const CompactCtx &K, cudaStream_t s);

}  // namespace lpp
