// round_dev.cuh -- the per-row and per-column work of one presolve round:
// S1 activities, S2 row classes, S3 implied bounds (fused, per row), S3'/S4
// bound finalisation and fixing (per column), S5 parallel rows (per row).
// Included by the round kernels (k_round.cu), which launch it over a whole
// arena, and by the fused batch kernel (k_batch.cu), which runs it for one
// LP per thread block: both evaluate every row and column the same way, so
// an LP gets the same bits from either.
#pragma once
#include <cooperative_groups.h>

#include "lpp_dev.cuh"

namespace lpp {

namespace {

namespace cg = cooperative_groups;

// appends v to list[*cnt ...] with one atomic per group of converged threads
__device__ __forceinline__ void coalesced_append(int32_t v, int32_t *cnt, int32_t *list) {
    cg::coalesced_group g = cg::coalesced_threads();
    int32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(cnt, (int32_t)g.size());
    base = g.shfl(base, 0);
    list[base + (int32_t)g.thread_rank()] = v;
}

// column j received a candidate: list it once per round for S3'
// (not needed when S3' checks every column this round)
__device__ __forceinline__ void touch_col(const Ctx &C, int32_t j) {
    if (!C.list_touched) {
        // a first round lists nothing (S3' runs on every column); with dual
        // records the flag alone lets the bound-source pass skip the columns
        // without a candidate
        if (C.dual_rec && C.ctouch[j] == 0u) C.ctouch[j] = 1u;
        return;
    }
    if (C.ctouch[j] == 0u && atomicExch(&C.ctouch[j], 1u) == 0u) coalesced_append(j, C.tl_cnt, C.tl_list);
}

// exact sign tests of a double on its bit pattern (integer pipes):
// s < 0 <=> negative and not -0;  s > 0 <=> positive bits, not +0
__device__ __forceinline__ bool lt0(double s) {
    return dbits(s) < 0 && dbits(s) != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool gt0(double s) { return dbits(s) > 0; }

// Implied upper bound x/a on column j (from a*x_j <= x with a > 0, or
// a*x_j >= x with a < 0).  Accepted iff (uold = +inf or x/a < thr) and
// |x/a| <= max_implied, thr = uold - bound_tol*max(1,|uold|) (one rounding).
// Both tests are decided exactly on the real quotient by the sign of one
// fused multiply-add; the cap is tested only for candidates that pass.
// A candidate that cannot lower the column's current minimum cur (x/a >= cur)
// would not change the result: it is dropped by the same test, made against
// min(cur, thr), and skips the divide.  pass_upper makes the sign test;
// apply_cand the cap, the divide and the atomic.
__device__ __forceinline__ bool pass_upper(const Ctx &C, int32_t j, double x, double a, double uold) {
    // x/a must lie below both cur and thr: one test against min(cur, thr),
    // taken on the order-preserving encoding (integer pipes)
    unsigned long long e = *((volatile unsigned long long *)&C.cand_u[j]);
    if (is_fin(uold)) {
        const unsigned long long et = enc_dbl(fma(-C.bound_tol, max1abs(uold), uold));
        e = et < e ? et : e;
    }
    if (e == kEncPosInf) return true;
    const double s = fma(-dec_dbl(e), a, x);
    return is_neg(a) ? gt0(s) : lt0(s);
}
// Implied lower bound x/a: accepted iff (lold = -inf or x/a > thr) and
// |x/a| <= max_implied, thr = lold + bound_tol*max(1,|lold|); a candidate
// that cannot raise the current maximum is dropped with it.
__device__ __forceinline__ bool pass_lower(const Ctx &C, int32_t j, double x, double a, double lold) {
    unsigned long long e = *((volatile unsigned long long *)&C.cand_l[j]);
    if (is_fin(lold)) {
        const unsigned long long et = enc_dbl(fma(C.bound_tol, max1abs(lold), lold));
        e = et > e ? et : e;
    }
    if (e == kEncNegInf) return true;
    const double s = fma(-dec_dbl(e), a, x);
    return is_neg(a) ? lt0(s) : gt0(s);
}

// candidate kinds: implied bounds (capped) and singleton-row bounds (not)
enum : int32_t { CQ_UPPER = 0, CQ_LOWER = 1, CQ_SING_UPPER = 2, CQ_SING_LOWER = 3 };

// the value x/a enters column j's candidates
__device__ __forceinline__ void apply_cand(const Ctx &C, int32_t j, double x, double a, int32_t kind) {
    if (kind < CQ_SING_UPPER && gt0(fma(-C.max_implied, fabs(a), fabs(x)))) return;
    const double v = x / a;
    if (!is_fin(v)) return;
    if (kind == CQ_UPPER || kind == CQ_SING_UPPER) atomic_min_dbl(&C.cand_u[j], v);
    else atomic_max_dbl(&C.cand_l[j], v);
    touch_col(C, j);
}

// Sign tests of the two implied bounds of one entry (S3).  dU = U - smin and
// dL = L - smax are the row's slacks: U - (min activity of the other
// entries) = dU + a*bmin when every term is finite, = dU when this entry is
// the one infinite term.  w1 / w2: a candidate x1/a (x2/a) of kind k1 (k2)
// passed and still needs the cap and the divide.
__device__ __forceinline__ void tighten_tests(const Ctx &C, int32_t j, double a, bool up_row, bool lo_row, double dU,
                                              double dL, int nmin, int nmax, bool &w1, double &x1, int32_t &k1,
                                              bool &w2, double &x2, int32_t &k2, int32_t &tested) {
    const double2 b = C.lu[j];
    const bool neg = is_neg(a);
    const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
    const bool fmn = is_fin(bmin), fmx = is_fin(bmax);
    if (up_row && (fmn ? nmin == 0 : nmin == 1)) {
        // a x_j <= U - (min activity of the other entries)
        tested++;
        x1 = fmn ? fma(a, bmin, dU) : dU;
        if (!neg) {
            k1 = CQ_UPPER;
            w1 = pass_upper(C, j, x1, a, b.y);
        } else {
            k1 = CQ_LOWER;
            w1 = pass_lower(C, j, x1, a, b.x);
        }
    }
    if (lo_row && (fmx ? nmax == 0 : nmax == 1)) {
        // a x_j >= L - (max activity of the other entries)
        tested++;
        x2 = fmx ? fma(a, bmax, dL) : dL;
        if (!neg) {
            k2 = CQ_LOWER;
            w2 = pass_lower(C, j, x2, a, b.x);
        } else {
            k2 = CQ_UPPER;
            w2 = pass_upper(C, j, x2, a, b.y);
        }
    }
}

// one entry, candidates applied at once (long rows: few of them tighten)
__device__ __forceinline__ void tighten_entry(const Ctx &C, int32_t j, double a, bool up_row, bool lo_row,
                                              double dU, double dL, int nmin, int nmax, int32_t &tested) {
    bool w1 = false, w2 = false;
    double x1 = 0.0, x2 = 0.0;
    int32_t k1 = 0, k2 = 0;
    tighten_tests(C, j, a, up_row, lo_row, dU, dL, nmin, nmax, w1, x1, k1, w2, x2, k2, tested);
    if (w1) apply_cand(C, j, x1, a, k1);
    if (w2) apply_cand(C, j, x2, a, k2);
}

// Per-warp queue of candidates that passed their sign tests.  The divide
// (and the cap, the atomic) then runs 32 candidates at a time, one per lane,
// instead of on the one or two lanes of a warp that produced a candidate in
// a step: on GB300 an FP64 instruction costs the pipe the same however many
// lanes are active.  Every lane of the warp must call cq_push / cq_flush.
struct CandQueue {
    double *x, *a;
    int32_t *j, *kind;
    int32_t n;  // items held, the same in every lane
};
constexpr int kQueueCap = 64;

__device__ __forceinline__ void cq_push(const Ctx &C, CandQueue &q, bool want, double x, double a, int32_t j,
                                        int32_t kind) {
    const unsigned b = __ballot_sync(0xffffffffu, want);
    if (b == 0u) return;
    const int lane = threadIdx.x & 31;
    if (want) {
        const int32_t p = q.n + __popc(b & ((1u << lane) - 1u));
        q.x[p] = x;
        q.a[p] = a;
        q.j[p] = j;
        q.kind[p] = kind;
    }
    q.n += __popc(b);
    if (q.n < 32) return;
    __syncwarp();
    apply_cand(C, q.j[lane], q.x[lane], q.a[lane], q.kind[lane]);
    const int32_t rest = q.n - 32;
    double rx = 0.0, ra = 0.0;
    int32_t rj = 0, rk = 0;
    if (lane < rest) {
        rx = q.x[32 + lane];
        ra = q.a[32 + lane];
        rj = q.j[32 + lane];
        rk = q.kind[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        q.x[lane] = rx;
        q.a[lane] = ra;
        q.j[lane] = rj;
        q.kind[lane] = rk;
    }
    __syncwarp();
    q.n = rest;
}

__device__ __forceinline__ void cq_flush(const Ctx &C, CandQueue &q) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (lane < q.n) apply_cand(C, q.j[lane], q.x[lane], q.a[lane], q.kind[lane]);
    q.n = 0;
}

// Per-warp queue of S3 tests: an entry side that qualifies (its row slack
// finite, the other terms finite or it the one infinite term) is queued
// with its coefficient a, the row slack, the bound of its own term and the
// bound it would tighten; the residual, the threshold and the sign test (the
// FP64 work) then run 32 tests at a time, and the passing candidates go on
// to the candidate queue.  flags: the candidate kind, | 4 if the entry's own
// term is finite (residual = slack + a * bnd, else the slack itself).
struct TestQueue {
    double *a, *slack, *bnd, *bold;
    int32_t *j, *flags;
    int32_t n;
};

__device__ __forceinline__ void tq_run(const Ctx &C, CandQueue &cq, bool have, double a, double slack, double bnd,
                                       double bold, int32_t j, int32_t flags) {
    bool w = false;
    double x = 0.0;
    const int32_t kind = flags & 3;
    if (have) {
        x = (flags & 4) ? fma(a, bnd, slack) : slack;
        w = kind == CQ_UPPER ? pass_upper(C, j, x, a, bold) : pass_lower(C, j, x, a, bold);
    }
    cq_push(C, cq, w, x, a, j, kind);
}

__device__ __forceinline__ void tq_push(const Ctx &C, TestQueue &q, CandQueue &cq, bool want, double a, double slack,
                                        double bnd, double bold, int32_t j, int32_t flags) {
    const unsigned b = __ballot_sync(0xffffffffu, want);
    if (b == 0u) return;
    const int lane = threadIdx.x & 31;
    if (want) {
        const int32_t p = q.n + __popc(b & ((1u << lane) - 1u));
        q.a[p] = a;
        q.slack[p] = slack;
        q.bnd[p] = bnd;
        q.bold[p] = bold;
        q.j[p] = j;
        q.flags[p] = flags;
    }
    q.n += __popc(b);
    if (q.n < 32) return;
    __syncwarp();
    const double ia = q.a[lane], isl = q.slack[lane], ibn = q.bnd[lane], ibo = q.bold[lane];
    const int32_t ij = q.j[lane], ifl = q.flags[lane];
    const int32_t rest = q.n - 32;
    double ra = 0.0, rs = 0.0, rb = 0.0, ro = 0.0;
    int32_t rj = 0, rf = 0;
    if (lane < rest) {
        ra = q.a[32 + lane];
        rs = q.slack[32 + lane];
        rb = q.bnd[32 + lane];
        ro = q.bold[32 + lane];
        rj = q.j[32 + lane];
        rf = q.flags[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        q.a[lane] = ra;
        q.slack[lane] = rs;
        q.bnd[lane] = rb;
        q.bold[lane] = ro;
        q.j[lane] = rj;
        q.flags[lane] = rf;
    }
    __syncwarp();
    q.n = rest;
    tq_run(C, cq, true, ia, isl, ibn, ibo, ij, ifl);
}

__device__ __forceinline__ void tq_flush(const Ctx &C, TestQueue &q, CandQueue &cq) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const bool have = lane < q.n;
    double ia = 0.0, isl = 0.0, ibn = 0.0, ibo = 0.0;
    int32_t ij = 0, ifl = 0;
    if (have) {
        ia = q.a[lane];
        isl = q.slack[lane];
        ibn = q.bnd[lane];
        ibo = q.bold[lane];
        ij = q.j[lane];
        ifl = q.flags[lane];
    }
    __syncwarp();
    q.n = 0;
    tq_run(C, cq, have, ia, isl, ibn, ibo, ij, ifl);
}

// S2: class of a row from its activities, first match wins: infeasible
// sides, infeasible activity, empty, redundant, singleton.  Returns false if
// the row proves the LP infeasible.
// Order-preserving integer key of a non-NaN double (-0 and +0 equal): the
// row tests compare keys on the integer pipes instead of the FP64 pipe.
__device__ __forceinline__ long long dkey(double x) {
    const long long b = dbits(x);
    if ((b & 0x7fffffffffffffffLL) == 0) return 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

__device__ __forceinline__ bool classify(const Ctx &C, double Lv, double Uv, int32_t len, double smin, double smax,
                                         int nmin, int nmax, uint8_t &kind) {
    const double ft = C.feas_tol;
    const bool Lf = is_fin(Lv), Uf = is_fin(Uv);
    kind = RK_KEPT;
    const double mL = max1abs(Lv), mU = max1abs(Uv);  // >= 1: their bits order like their values
    if (Lf && Uf) {
        const double d = ft * (dbits(mL) > dbits(mU) ? mL : mU);
        if (dkey(Lv - Uv) > dkey(d)) return false;
    }
    const double uhi = Uv + ft * mU, llo = Lv - ft * mL;  // U + delta(U), L - delta(L)
    const long long ksmin = dkey(smin), ksmax = dkey(smax);
    if (nmin == 0 && Uf && ksmin > dkey(uhi)) return false;
    if (nmax == 0 && Lf && ksmax < dkey(llo)) return false;
    if (len == 0) {
        kind = RK_EMPTY;
        return true;
    }
    const bool lo_ok = !Lf || (nmin == 0 && ksmin >= dkey(llo));
    if (lo_ok) {
        const bool hi_ok = !Uf || (nmax == 0 && ksmax <= dkey(uhi));
        if (hi_ok) {
            kind = RK_REDUNDANT;
            return true;
        }
    }
    if (len == 1) kind = RK_SINGLETON;
    return true;
}


// writes the row's S1/S2 results and records; a singleton row returns its
// entry (sa, sj) for the caller to apply as bounds L/a, U/a
__device__ __forceinline__ int32_t finish_row(const Ctx &C, int32_t i, int32_t beg, int32_t len, double Lv,
                                              double Uv, double smin, double smax, int nmin, int nmax,
                                              unsigned long long h, uint8_t &kind, double &sa, int32_t &sj) {
    const bool ok = classify(C, Lv, Uv, len, smin, smax, nmin, nmax, kind);
    C.act[i] = make_double2(smin, smax);
    C.ninf[i] = make_int2(nmin, nmax);
    C.hrow[i] = h;
    const int32_t lp = lp_of_row(C, i);
    if (!ok) {
        atomicMin(&C.verdict[lp * V_SLOTS + V_S2_ROW], C.rmap[i]);
        kind = RK_KEPT;
        C.rkind[i] = RK_KEPT;
        return 0;
    }
    C.rkind[i] = kind;
    if (kind == RK_KEPT) return 0;
    const int32_t o = C.rmap[i];
    C.rec_rk[o] = kind;
    C.rec_rr[o] = lp_round(C, lp);
    mark_lp_changed(C, lp);
    if (kind == RK_SINGLETON) {
        // L <= a x_j <= U becomes a bound on x_j, always applied (no threshold)
        sa = C.A.val[beg];
        sj = C.A.idx[beg];
        C.rec_ra[o] = C.cmap[sj];
        C.rec_rv[o] = sa;
    } else {
        C.rec_ra[o] = -1;
        C.rec_rv[o] = 0.0;
    }
    return 1;
}

// ------------------------------------------------------- S1 + S2 + S3 groups
template <int W>
__device__ __forceinline__ void prop_group(const Ctx &C, int32_t i, bool valid, int32_t &removed, int32_t &evaluated,
                                           int32_t &tested, CandQueue &q, TestQueue &tq) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    // A row none of whose bounds, entries or sides changed since its last
    // evaluation has the same activities and class (kept) and yields the same
    // implied bounds, which were then already applied or rejected: skip it
    // (its lanes stay for the warp's queue steps).  Flag 2: such a row whose
    // columns were renumbered by a compaction since; only its S5 key, which
    // hashes the column indices, is taken again (no bound gathers).
    const uint8_t flag = valid ? C.rdirty[i] : 0;
    const bool act = flag == 1, rehash = flag == 2;
    if (valid && !act && lane == 0) C.rkind[i] = RK_KEPT;
    int32_t beg = 0, end = 0;
    if (act || rehash) {
        beg = C.A.ptr[i];
        end = C.A.ptr[i + 1];
    }
    const bool neg0 = end > beg ? is_neg(C.A.val[beg]) : false;
    double smin = 0.0, smax = 0.0;
    int nmin = 0, nmax = 0;
    unsigned long long h = 0;
    // The lane's entries in steps of four, the tail of a step predicated: the
    // four bound gathers of a step overlap, and a warp whose lanes hold rows of
    // different lengths runs no separate remainder loop (which would issue
    // its FP64 work a second time for the lanes still in it).  The sums take
    // the entries in the same order as a plain loop.
    for (int32_t k0 = beg + lane; k0 < end; k0 += 4 * W) {
        int32_t jq[4];
        double aq[4];
        double2 bq[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int32_t k = k0 + q * W;
            jq[q] = k < end ? C.A.idx[k] : 0;
            aq[q] = k < end ? C.A.val[k] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) bq[q] = act && k0 + q * W < end ? C.lu[jq[q]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (k0 + q * W >= end) break;
            const double a = aq[q];
            const double2 b = bq[q];
            const bool neg = is_neg(a);
            const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
            if (is_fin(bmin)) smin = fma(a, bmin, smin);
            else nmin++;
            if (is_fin(bmax)) smax = fma(a, bmax, smax);
            else nmax++;
            h += entry_hash(jq[q], neg != neg0);
        }
    }
    smin = group_sum<W>(smin, mask);
    smax = group_sum<W>(smax, mask);
    nmin = group_sum<W>(nmin, mask);
    nmax = group_sum<W>(nmax, mask);
    h = group_sum<W>(h, mask);
    const int32_t len = end - beg;
    if (rehash && lane == 0) C.hrow[i] = h + len_hash(len);
    bool up_row = false, lo_row = false;
    double dU = 0.0, dL = 0.0, Lv = 0.0, Uv = 0.0, sa = 0.0;
    int32_t sj = -1;
    if (act) {
        h += len_hash(len);
        if (lane == 0) evaluated += len;
        Lv = C.L[i];
        Uv = C.U[i];
        uint8_t kind = RK_KEPT;
        if (lane == 0) removed += finish_row(C, i, beg, len, Lv, Uv, smin, smax, nmin, nmax, h, kind, sa, sj);
        kind = (uint8_t)__shfl_sync(mask, (int)kind, 0, W);
        if (kind == RK_KEPT && len >= 2) {
            up_row = is_fin(Uv) && nmin <= 1;
            lo_row = is_fin(Lv) && nmax <= 1;
            dU = Uv - smin;
            dL = Lv - smax;
        }
    }
    // a singleton row's bounds L/a and U/a (a < 0 swaps them)
    const bool sing = sj >= 0, sneg = is_neg(sa);
    cq_push(C, q, sing && is_fin(Lv), Lv, sa, sj, sneg ? CQ_SING_UPPER : CQ_SING_LOWER);
    cq_push(C, q, sing && is_fin(Uv), Uv, sa, sj, sneg ? CQ_SING_LOWER : CQ_SING_UPPER);
    // S3 over the row's entries, in steps the whole warp takes together
    const int32_t trips = (up_row || lo_row) && lane < len ? (len - lane + W - 1) / W : 0;
    const int32_t T = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)trips);
    for (int32_t it = 0; it < T; it++) {
        bool w1 = false, w2 = false;
        double a = 0.0, bn1 = 0.0, bn2 = 0.0, bo1 = 0.0, bo2 = 0.0;
        int32_t j = 0, f1 = 0, f2 = 0;
        if (it < trips) {
            const int32_t k = beg + lane + it * W;
            j = C.A.idx[k];
            a = C.A.val[k];
            const double2 b = C.lu[j];
            const bool neg = is_neg(a);
            const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
            const bool fmn = is_fin(bmin), fmx = is_fin(bmax);
            if (up_row && (fmn ? nmin == 0 : nmin == 1)) {  // a x_j <= U - (min activity of the others)
                w1 = true;
                bn1 = bmin;
                bo1 = neg ? b.x : b.y;
                f1 = (neg ? CQ_LOWER : CQ_UPPER) | (fmn ? 4 : 0);
            }
            if (lo_row && (fmx ? nmax == 0 : nmax == 1)) {  // a x_j >= L - (max activity of the others)
                w2 = true;
                bn2 = bmax;
                bo2 = neg ? b.y : b.x;
                f2 = (neg ? CQ_UPPER : CQ_LOWER) | (fmx ? 4 : 0);
            }
            tested += (w1 ? 1 : 0) + (w2 ? 1 : 0);
        }
        tq_push(C, tq, q, w1, a, dU, bn1, bo1, j, f1);
        tq_push(C, tq, q, w2, a, dL, bn2, bo2, j, f2);
    }
}

// Lanes per row in S1-S3: one thread per row up to 16 entries (the row's
// classification then runs on every lane of the warp), else the class width.
__host__ __device__ __forceinline__ int prop_lanes(int c) { return c <= 2 ? 1 : 1 << c; }

// ------------------------------------------------- S3' finalise + S4 fixing
// S3' + S4 on column j: apply the accepted candidates, check and snap the
// bounds, fix the column if l == u.  Adds to the counts changed, fixed and
// chg_nnz (a thread may finalise several columns); a changed short column is
// listed for the dirty-row marking.
__device__ __forceinline__ void colfin_one(const Ctx &C, int32_t j, bool full, int32_t &changed, int32_t &fixed,
                                           int32_t &chg_nnz) {
    const unsigned long long el = C.cand_l[j], eu = C.cand_u[j];
    const bool has = el != kEncNegInf || eu != kEncPosInf;
    uint8_t kind = CK_KEPT;
    uint8_t chg = 0;
    const int32_t lp = lp_of_col(C, j);
    if (has || (full && lp_round(C, lp) == 1)) {
        if (has) {
            C.cand_l[j] = kEncNegInf;
            C.cand_u[j] = kEncPosInf;
        }
        const double2 b = C.lu[j];
        double nl = b.x, nu = b.y;
        if (has) {
            const double dl = dec_dbl(el), du = dec_dbl(eu);
            if (dl > nl) nl = dl;
            if (du < nu) nu = du;
        }
        bool bad = false;
        if (is_fin(nl) && is_fin(nu)) {
            const double d = C.feas_tol * fmax(1.0, fmax(fabs(nl), fabs(nu)));
            if (nl - nu > d) {
                bad = true;
            } else if (nl != nu && fabs(nl - nu) <= d) {
                const double mid = 0.5 * (nl + nu);
                nl = mid;
                nu = mid;
            }
        }
        if (bad) {
            atomicMin(&C.verdict[lp * V_SLOTS + V_S3_COL], C.cmap[j]);
        } else {
            if (C.dual_rec && has) {
                // a side a candidate moved takes that candidate's row (a side
                // moved only by the snap keeps its earlier source)
                const int2 src = C.bsrc[j];
                const double dl = dec_dbl(el), du = dec_dbl(eu);
                if (dl > b.x || du < b.y) {
                    int4 r = C.rec_bs[C.cmap[j]];
                    if (dl > b.x) {
                        r.x = src.x != INT32_MAX ? src.x : -2;  // -2: no row matched (never expected)
                        r.y = lp_round(C, lp);
                    }
                    if (du < b.y) {
                        r.z = src.y != INT32_MAX ? src.y : -2;
                        r.w = lp_round(C, lp);
                    }
                    C.rec_bs[C.cmap[j]] = r;
                }
                C.bsrc[j] = make_int2(INT32_MAX, INT32_MAX);
            }
            if (nl != b.x || nu != b.y) {
                C.lu[j] = make_double2(nl, nu);
                changed++;
                chg = 1;
                mark_lp_changed(C, lp);
            }
            if (nl == nu) {
                kind = CK_FIXED;
                fixed++;
                C.fixv[j] = nl;
                const int32_t o = C.cmap[j];
                C.rec_ck[o] = CK_FIXED;
                C.rec_cr[o] = lp_round(C, lp);
                C.rec_cv[o] = nl;
                mark_lp_changed(C, lp);
            }
        }
    }
    C.ckind[j] = kind;
    C.cchg[j] = chg;
    C.ctouch[j] = 0u;
    if (chg) {
        // the column's segment in T (input numbering when T is not compacted)
        // decides list or chunks for the dirty-row marking; its current
        // entries count towards the marking threshold
        const int32_t jt = C.t_orig ? C.cmap[j] : j;
        const int32_t len = C.T.ptr[jt + 1] - C.T.ptr[jt];
        if (len < kLongMin) coalesced_append(j, C.cl_cnt, C.cl_list);
        chg_nnz += C.t_orig ? C.clen[j] : len;
    }
}

// ------------------------------------------------------------ S5 parallel rows
// Inserts row i into the hash table of capacity cap (a power of two) and
// elects the leader of its key: the first equality row, else the first row
// (Sec. 3.2), by atomicMin on (is_ineq, row).  Returns the slot, -1 if the
// table is full (an internal error: the capacity is at least twice the rows).
__device__ __forceinline__ int32_t s5_insert_row(const Ctx &C, int32_t i, uint32_t cap) {
    unsigned long long key = C.hrow[i];
    if (key == 0) key = 1;
    uint32_t sl = (uint32_t)(key ^ (key >> 32)) & (cap - 1u);
    for (uint32_t probe = 0; probe < cap; probe++) {
        const unsigned long long prev = atomicCAS(&C.tkey[sl], 0ULL, key);
        if (prev == 0ULL || prev == key) {
            const double Lv = C.L[i], Uv = C.U[i];
            const bool eq = is_fin(Lv) && Lv == Uv;
            const unsigned long long code = ((unsigned long long)(eq ? 0u : 1u) << 32) | (uint32_t)i;
            atomicMin(&C.tlead[sl], code);
            return (int32_t)sl;
        }
        sl = (sl + 1u) & (cap - 1u);
    }
    atomicOr(&C.st->err, 1);
    return -1;
}

// merge a parallel follower i (row = lam * leader) into its leader li
__device__ __forceinline__ void s5_accept(const Ctx &C, int32_t i, int32_t li, double lam) {
    C.rkind[i] = RK_PARALLEL;
    const int32_t o = C.rmap[i];
    const int32_t lp = lp_of_row(C, i);
    C.rec_rk[o] = RK_PARALLEL;
    C.rec_rr[o] = lp_round(C, lp);
    C.rec_ra[o] = C.rmap[li];
    C.rec_rv[o] = lam;
    mark_lp_changed(C, lp);
    const double Lj = C.L[i], Uj = C.U[i];
    double lo, hi;
    if (!is_neg(lam)) {
        lo = is_fin(Lj) ? Lj / lam : ninf_();
        hi = is_fin(Uj) ? Uj / lam : pinf();
    } else {
        lo = is_fin(Uj) ? Uj / lam : ninf_();
        hi = is_fin(Lj) ? Lj / lam : pinf();
    }
    if (is_fin(lo)) atomic_max_dbl(&C.mL[li], lo);
    if (is_fin(hi)) atomic_min_dbl(&C.mU[li], hi);
    C.hasf[li] = 1;
}

template <int W>
__device__ __forceinline__ bool match_group(const Ctx &C, int32_t i, bool valid, int32_t &removed,
                                            int32_t &unmatched) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    bool act = valid && C.rwork[i] == 1;
    int32_t li = -1;
    if (act) {
        li = (int32_t)(uint32_t)(C.tlead[C.rslot[i]] & 0xffffffffULL);
        if (li == i) act = false;  // the leader itself
    }
    // every lane of a group sees the same `act`
    int32_t bi = 0, bl = 0, len = 0;
    bool ok = false;
    double lam = 0.0;
    if (act) {
        bi = C.A.ptr[i];
        bl = C.A.ptr[li];
        len = C.A.ptr[i + 1] - bi;
        ok = (C.A.ptr[li + 1] - bl) == len;
        lam = C.A.val[bi] / C.A.val[bl];
    }
    if (ok) {
        for (int32_t k = lane; k < len; k += W) {
            const double ai = C.A.val[bi + k], al = C.A.val[bl + k];
            const double la = lam * al;
            const bool same = C.A.idx[bi + k] == C.A.idx[bl + k] &&
                              fabs(ai - la) <= C.par_tol * fmax(fabs(ai), fabs(la));
            if (!same) ok = false;
        }
    }
    // all lanes of the group agree on `ok`
    const unsigned bal = __ballot_sync(mask, !ok);
    const unsigned mine = group_bits<W>(bal);
    ok = act && mine == 0u;
    if (valid && lane == 0) {
        if (ok) {
            s5_accept(C, i, li, lam);
            C.rwork[i] = 0;
            removed++;
        } else if (act) {
            C.rwork[i] = 2;
            unmatched++;
        } else {
            C.rwork[i] = 0;
        }
    }
    return valid && lane == 0 && act && !ok;
}

// table capacity of a later pass over n listed rows: the power of two >= 2 n, at most C.tcap
__device__ __forceinline__ uint32_t s5_tail_cap(const Ctx &C, int32_t n) {
    uint32_t cap = 1;
    while (cap < 2u * (uint32_t)n && cap < (uint32_t)C.tcap) cap <<= 1;
    return cap;
}

// Later-pass match of entry t of a list of n rows (t >= n: no row): row i
// against the leader of its slot; rows longer than 32 entries are checked
// by the whole warp in turn, so every lane of the warp must call it.
// removed / left: the row merged, or left unmatched for the next pass.
__device__ __forceinline__ void s5_tail_match_one(const Ctx &C, const int32_t *list, int32_t n, int32_t t,
                                                  int32_t &removed, bool &left, int32_t &i) {
    removed = 0;
    left = false;
    i = -1;
    const int lane = threadIdx.x & 31;
    bool act = false, ok = false;
    int32_t li = -1, bi = 0, bl = 0, len = 0;
    double lam = 0.0;
    if (t < n) {
        // the list, the slots and the leaders change from pass to pass, also
        // within one launch (grid-wide passes): read at L2, never from L1
        i = __ldcg(list + t);
        const int32_t sl = __ldcg(C.rslot + i);
        act = sl >= 0;
        if (act) {
            li = (int32_t)(uint32_t)(__ldcg(C.tlead + sl) & 0xffffffffULL);
            if (li == i) act = false;  // the leader itself
        }
        if (act) {
            bi = C.A.ptr[i];
            bl = C.A.ptr[li];
            len = C.A.ptr[i + 1] - bi;
            ok = (C.A.ptr[li + 1] - bl) == len;
            lam = C.A.val[bi] / C.A.val[bl];
        }
    }
    if (ok && len <= 32) {
        for (int32_t k = 0; k < len; k++) {
            const double ai = C.A.val[bi + k], la = lam * C.A.val[bl + k];
            if (!(C.A.idx[bi + k] == C.A.idx[bl + k] && fabs(ai - la) <= C.par_tol * fmax(fabs(ai), fabs(la)))) {
                ok = false;
                break;
            }
        }
    }
    unsigned todo = __ballot_sync(0xffffffffu, ok && len > 32);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int32_t sbi = __shfl_sync(0xffffffffu, bi, src), sbl = __shfl_sync(0xffffffffu, bl, src);
        const int32_t slen = __shfl_sync(0xffffffffu, len, src);
        const double slam = __shfl_sync(0xffffffffu, lam, src);
        bool sok = true;
        for (int32_t k = lane; k < slen; k += 32) {
            const double ai = C.A.val[sbi + k], la = slam * C.A.val[sbl + k];
            if (!(C.A.idx[sbi + k] == C.A.idx[sbl + k] && fabs(ai - la) <= C.par_tol * fmax(fabs(ai), fabs(la))))
                sok = false;
        }
        sok = __all_sync(0xffffffffu, sok) != 0;
        if (lane == src) ok = sok;
    }
    if (act && ok) {
        s5_accept(C, i, li, lam);
        removed = 1;
    } else if (act) {
        left = true;
    }
}

// leaders take the followers' sides: L = max(L, merged), U = min(U, merged);
// crossing by more than the tolerance is infeasible, nearly equal sides snap
// (row i has followers: hasf[i])
__device__ __forceinline__ void s5_leader_one(const Ctx &C, int32_t i) {
    C.hasf[i] = 0;
    const unsigned long long eL = C.mL[i], eU = C.mU[i];
    C.mL[i] = kEncNegInf;
    C.mU[i] = kEncPosInf;
    double nL = C.L[i], nU = C.U[i];
    const double mL = dec_dbl(eL), mU = dec_dbl(eU);
    if (mL > nL) nL = mL;
    if (mU < nU) nU = mU;
    if (is_fin(nL) && is_fin(nU)) {
        const double d = C.feas_tol * fmax(1.0, fmax(fabs(nL), fabs(nU)));
        if (nL - nU > d) {
            atomicMin(&C.verdict[lp_of_row(C, i) * V_SLOTS + V_S5_ROW], C.rmap[i]);
            return;
        }
        if (nL != nU && fabs(nL - nU) <= d) {
            const double mid = 0.5 * (nL + nU);
            nL = mid;
            nU = mid;
        }
    }
    if (nL != C.L[i] || nU != C.U[i]) C.rdnext[i] = 1;
    C.L[i] = nL;
    C.U[i] = nU;
}

}  // namespace

}  // namespace lpp
