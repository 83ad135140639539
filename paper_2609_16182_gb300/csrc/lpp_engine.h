// lpp_engine.h -- the presolve engine behind the C ABI (internal).
//
// One Engine owns the device state of an "arena": one LP (plain mode) or many
// LPs laid out back to back as one block-diagonal LP (batch and serving).
// Every kernel sees the arena as a single LP; per-LP bookkeeping (verdicts,
// rounds, objective constant) uses lp_row / lp_col.  Because a row's or a
// column's arithmetic never depends on its neighbours, an LP's result in an
// arena equals its result alone.
#pragma once
#include <cstdint>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/lpp.h"
#include "lpp_launch.h"

namespace lpp {

struct CudaError : std::runtime_error {
    cudaError_t code;
    CudaError(cudaError_t c, const std::string &what) : std::runtime_error(what), code(c) {}
};
struct StatusError : std::runtime_error {
    lpp_status st;
    StatusError(lpp_status s, const std::string &what) : std::runtime_error(what), st(s) {}
};

void cuda_check(cudaError_t e, const char *expr, const char *file, int line);
#define LPP_CUDA(x) ::lpp::cuda_check((x), #x, __FILE__, __LINE__)

// A process-wide cache of device blocks that finished presolves released,
// by device and exact size: a presolve makes some seventy allocations, and
// the next presolve of an LP of the same sizes takes them back without a
// call into the allocator.  take: such a block, or nullptr.
void *dev_cache_take(size_t bytes);
void dev_cache_put(void *p, size_t bytes, cudaStream_t s);

// stream-ordered device allocations released together (to the cache, once
// the stream's work on them is done)
struct DevPool {
    cudaStream_t s = nullptr;
    bool cache = true;  // false: released stream-ordered, without a wait
    std::vector<void *> ptrs;
    std::vector<size_t> sizes;
    template <class T>
    T *alloc(size_t cnt) {
        const size_t bytes = (cnt ? cnt : 1) * sizeof(T);
        void *p = dev_cache_take(bytes);
        if (!p) LPP_CUDA(cudaMallocAsync(&p, bytes, s));
        ptrs.push_back(p);
        sizes.push_back(bytes);
        return static_cast<T *>(p);
    }
    void forget(void *p);  // ownership moves elsewhere
    void release();
    ~DevPool() { release(); }
};

// per-LP description of an arena member
struct Member {
    int32_t m, n;
    int64_t nnz;
    int32_t row_off, col_off;
    int64_t nnz_off;
    double obj_offset;
};

// Device buffers and host mirror of one arena.
struct Engine {
    lpp_opts o;
    cudaStream_t s = nullptr;
    bool own_stream = false;
    DevPool pool;
    int32_t nlp = 1;
    std::vector<Member> mem;
    int32_t m0 = 0, n0 = 0;
    int64_t nnz0 = 0;
    // current sizes
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    int cur = 0;
    // double buffers
    int32_t *rp[2], *ci[2], *tp[2], *ti[2];
    double *rv[2], *tv[2];
    double *L[2], *U[2], *c[2];
    double2 *lu[2];
    int32_t *rmap[2], *cmap[2], *lprow[2], *lpcol[2];
    // schedules
    SchedBufs sa, sb;  // A (rows), T (columns)
    int32_t cap_long_a, cap_long_t;
    // work (row results are double-buffered: clean rows carry them over)
    double2 *act[2];
    int2 *ninf[2];
    unsigned long long *hrow[2];
    uint8_t *rdirty[2], *rdnext, *cchg;
    uint8_t *rkind, *rwork, *hasf, *ckind, *lneed, *lp_changed, *lp_dead;
    unsigned long long *mL, *mU, *cand_l, *cand_u, *tkey, *tlead, *ch_hash;
    int32_t *s5_list[2] = {nullptr, nullptr}, *s5_cnt = nullptr;
    unsigned *s5_bar = nullptr;  // grid barrier of the cooperative S5 passes (two words)
    bool s5_clean = false;  // the last S5 resolved every group and no row changed since
    // S5c (opts.parallel_cols): slots and the column table; flags, positions
    // and the (slot, column) pairs of the grouped columns with their sort
    // buffers; per-position cached data and live flags; the large groups
    unsigned long long *ctkey = nullptr;
    int32_t *cslot = nullptr, *ctcnt = nullptr, *ctnew = nullptr, *pc_cnt = nullptr, *pcnt = nullptr, *plen = nullptr;
    unsigned long long *pkey = nullptr;
    void *pc_mem = nullptr;
    int32_t *pc_flags = nullptr, *pc_pos = nullptr, *pc_col = nullptr, *pc_scan = nullptr;
    uint32_t *pc_slot = nullptr;
    TransposeBufs pc_sort{};
    uint8_t *pc_alive = nullptr;
    int2 *pc_glist = nullptr;
    int32_t ctcap_max = 0;
    bool s5c_dirty = true;   // a row was removed or a column fixed or merged since the last S5c
    // S5d (opts.col_singletons): candidate per row, eligibility per row, the
    // first eligible row per column, the long rows deferred to block tasks
    int32_t *cs_rcand = nullptr, *cs_cmin = nullptr, *cs_tasks = nullptr, *cs_ntask = nullptr;
    uint8_t *cs_relig = nullptr;
    double *cs_a = nullptr;  // per row: the candidate's coefficient (rows of more than 4096 entries)
    // S5e (opts.doubletons): the step's work (see S5eBufs), a pinned copy of
    // its two counts, the transpose histogram kept from the ingest
    S5eBufs de{};
    int32_t *de_cnt_h = nullptr;
    int32_t *t_hist = nullptr;
    cudaStream_t s2 = nullptr;                   // host inputs: the vectors' copies
    cudaStream_t s_long = nullptr;               // the long rows' kernels (S1-S3, row counts), beside
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // the short rows' kernel
    void ensure_side_stream();
    cudaEvent_t ev_mat = nullptr, ev_vec = nullptr;
    bool vec_pending = false;                    // their check waits for the copies (prepare)
    uint32_t *ctouch = nullptr;                                      // S3' column lists
    int32_t *tl_list = nullptr, *cl_list = nullptr, *col_cnt = nullptr;  // S5 lists of unmatched rows, their sizes per pass
    int32_t *rslot, *verdict;
    double *fixv;
    double2 *ch_act;
    int2 *ch_ninf;
    int32_t tcap_max;
    // The CSC kept as the input's A^T and the columns kept in place instead
    // of compacted each round (set by setup when lazy_req and no step that
    // reads columns' entries is on): input-to-current row map, column map
    // (the slot itself while the column is in the LP, -1 once it left),
    // entries per column in the current rows, and at the end the input rows
    // still in the LP (columns and CSC are compacted once, at the end).
    bool lazy_req = false, t_orig = false, t_fixed = false;
    int32_t *rinv = nullptr, *cinv = nullptr, *clive = nullptr;
    uint8_t *rleft = nullptr;
    void finish_cols();  // the columns' one compaction (t_orig)
    // opts.dep_rows: the equality rows' dependencies found on the host and
    // the rows removed by one more compaction (single LP)
    void remove_dependent();
    double2 *act_rec = nullptr;  // the last round's activities and row map when that step's
    int2 *ninf_rec = nullptr;    // compaction had to write over their buffers
    int32_t *rmap_rec = nullptr;
    int64_t dep_pivots = 0, dep_peeled = 0;
    int32_t dep_found = 0, dep_stopped = 0;
    void finish_csc();   // the result's CSC from the input's (t_orig)
    // compaction work
    CompactCtx K;
    int32_t *scan_tmp;
    // records
    int32_t *rec_rk, *rec_rr, *rec_ra, *rec_ck, *rec_cr;
    double *rec_rv, *rec_cv;
    int32_t *rec_ca = nullptr, *rec_cp = nullptr;  // S5c merges (NULL unless opts.parallel_cols)
    double *rec_cm = nullptr;
    long long *rec_sb = nullptr;                   // S5d / S5e substitutions (NULL unless opts.col_singletons
                                                   // or opts.doubletons)
    int32_t *rec_sl = nullptr, *rec_scol = nullptr;
    double *rec_srhs = nullptr, *rec_sval = nullptr;
    unsigned long long *sub_used = nullptr;
    int4 *rec_bs = nullptr;                         // bound sources (NULL unless opts.dual_records):
    int2 *bsrc = nullptr;                           // per original column, and this round's per column
    DevStatus *st;
    DevStatus *st_h = nullptr;  // pinned mirror
    int32_t *verdict_h = nullptr;
    uint8_t *changed_h = nullptr;
    int32_t *s5_left_h = nullptr;  // rows still unmatched after a chunk of S5 passes
    SegMat A, T;
    // per-LP results
    std::vector<int32_t> lp_rounds, lp_status, lp_where, lp_index, lp_round;
    std::vector<uint8_t> lp_done;
    // per-round statistics
    std::vector<int64_t> r_nnz;
    std::vector<int32_t> r_rows, r_cols, r_bounds;
    std::vector<float> r_ms;
    int32_t rounds = 0;
    double loop_ms = 0.0;
    int64_t nnz_processed = 0;
    int64_t s5_left = 0;    // rows unmatched when the S5 leader passes stopped at the cap, summed over rounds
    int64_t launches0 = 0;  // launch counter at setup
    // activities of the last round: current-index arrays and the map valid then
    int32_t act_m = 0, act_buf = 0;
    // kernel timing
    struct Tmark {
        int fam;
        cudaEvent_t a, b;
        double bytes, ops;
    };
    std::vector<int64_t> r_eval;  // nonzeros S1 evaluated per round
    std::vector<Tmark> marks;
    std::vector<cudaEvent_t> spare_events;

    ~Engine();
    void setup(const lpp_opts &opts, int32_t nlp_, const std::vector<Member> &members);
    // ingest: the LPs' arrays are copied into the arena and checked
    void ingest_plain(const lpp_lp &in);
    void ingest_batch(const lpp_lp *ins, int32_t count);
    void prepare();  // after ingest: transpose, schedules, work init
    void run();      // the round loop
    struct StepOut {
        bool structural = false;
        float ms = 0.f;
    };
    StepOut step(int32_t r, bool first_round, bool force);
    // serving: an empty arena that LPs join and leave between rounds
    int32_t *lp_round0_dev = nullptr;
    uint8_t *lp_retired_dev = nullptr;
    void init_empty();
    void append(int32_t slot, const lpp_lp &in, int32_t rbase, int32_t cbase, int32_t round0);
    void reschedule();
    void k_sizes_set(int32_t m_, int32_t n_);
    cudaEvent_t ev_round[2] = {nullptr, nullptr};
    std::vector<uint8_t> lp_dropped;
    Ctx ctx(int32_t round) const;
    void read_status();
    void schedule_current();
    void adopt_schedule();
    void compact(int32_t round);
    void run_s5c(const Ctx &C0);  // S5c: keys, the changed groups, their leader passes
    void run_s5d(const Ctx &C);   // S5d: column singletons, then a status read
    void run_s5e(const Ctx &C);   // S5e: doubleton equations, the rewritten matrices, a status read
    // timing helpers
    void tbegin(int fam, double bytes);
    void tend();
};

// Kernel families reported by lpp_result_kernels.
enum Fam {
    F_PROP = 0, F_COLFIN, F_S5, F_COUNT, F_SCAN, F_SCATTER, F_SCHED, F_INGEST, F_FINISH, F_S5C, F_S5D, F_S5E, F_NUM
};
const char *fam_name(int f);

// device allocations shared by the reduced LPs of one batch, freed with the last
struct SharedStore {
    std::vector<void *> ptrs;
    ~SharedStore() {
        for (void *p : ptrs) cudaFree(p);
    }
};

}  // namespace lpp

// sets the message lpp_last_error() returns and passes the status through
lpp_status lpp_noalloc_fail(lpp_status st, const char *msg);

namespace lpp {
// pinned host buffers from a process-wide cache (first fit by capacity)
void *pinned_get_sized(size_t bytes);
void pinned_put(void *p);
}  // namespace lpp

// Library objects behind the opaque C handles.
struct lpp_reduced {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    double obj_offset = 0.0;
    int32_t *rp = nullptr, *ci = nullptr, *tp = nullptr, *ti = nullptr, *rmap = nullptr, *cmap = nullptr;
    double *rv = nullptr, *tv = nullptr, *L = nullptr, *U = nullptr, *lb = nullptr, *ub = nullptr, *c = nullptr;
    std::vector<void *> owned;  // device allocations
    std::shared_ptr<lpp::SharedStore> shared;  // batch: storage shared with the other LPs
    // host copies made on the first request for them (on_device = 0), into
    // one pinned block
    void *hblock = nullptr;
    int host_done = 0;  // groups copied: 1 = LP, 2 = maps, 4 = CSC
    int32_t *h_rp = nullptr, *h_ci = nullptr, *h_tp = nullptr, *h_ti = nullptr, *h_rmap = nullptr, *h_cmap = nullptr;
    double *h_rv = nullptr, *h_c = nullptr, *h_L = nullptr, *h_U = nullptr, *h_lb = nullptr, *h_ub = nullptr,
           *h_tv = nullptr;
};

namespace lpp {
// Device-resident results of one engine run (all its LPs), shared by their
// postsolve records; the host copies are made on first access.
struct DeviceRecords {
    int32_t m0 = 0, n0 = 0, n_final = 0, act_m = 0;
    int32_t *rk = nullptr, *rr = nullptr, *ra = nullptr, *ck = nullptr, *cr = nullptr;
    double *rv = nullptr, *cv = nullptr;
    int32_t *ca = nullptr, *cp = nullptr;  // S5c merges: leader, pass (NULL without parallel_cols)
    double *cm = nullptr;                  // [4 per column] bounds at the merge
    long long *sb = nullptr;               // S5d substitutions (NULL without col_singletons)
    int32_t *sl = nullptr, *scol = nullptr;
    double *srhs = nullptr, *sval = nullptr;
    int64_t sub_used = 0;                  // entries in the store
    int4 *bs = nullptr;                    // bound sources (NULL without dual_records)
    std::once_flag store_once;             // the host copy of the store, made once
    std::vector<int32_t> h_scol;
    std::vector<double> h_sval;
    double2 *lu = nullptr;       // [n_final] final bounds of the kept columns (arena order)
    int32_t *cmap = nullptr;     // [n_final] their original (arena) index
    double2 *act = nullptr;      // [act_m] last round's activities (that round's numbering)
    int2 *ninf = nullptr;
    int32_t *act_rmap = nullptr;
    std::vector<void *> owned;
    ~DeviceRecords() {
        for (void *p : owned) cudaFree(p);
    }
};
}  // namespace lpp

struct lpp_postsolve {
    lpp_info info{};
    std::shared_ptr<lpp::DeviceRecords> dev;
    double huge = 1e20;              // opts.huge of the presolve (infinite sides of the input LP)
    int32_t r0 = 0, c0 = 0;          // first original row / column of this LP in the arena
    int32_t cstart = 0;              // first kept column of this LP in the final arena
    int32_t astart = 0, acnt = 0;    // this LP's rows in the last round's numbering
    bool host_ready = false;
    std::vector<int32_t> row_kind, row_round, row_aux, col_kind, col_round, col_map, col_aux, col_pass;
    std::vector<double> row_val, col_val, col_lb, col_ub, act_min, act_max, col_mrg;
    std::vector<int64_t> sub_beg;                 // substitutions: per row, into sub_col / sub_val
    std::vector<int32_t> sub_len, sub_col;
    std::vector<double> sub_rhs, sub_val;
    std::vector<int32_t> ninf_min, ninf_max;
    std::vector<int32_t> col_lsrc, col_lrnd, col_usrc, col_urnd;  // bound sources (empty without them)
    std::vector<int64_t> r_nnz;
    std::vector<int32_t> r_rows, r_cols, r_bounds;
    std::vector<float> r_ms;
    std::vector<lpp_kernel_stat> kstats;
};
