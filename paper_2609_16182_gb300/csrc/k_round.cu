// k_round.cu -- the kernels of one presolve round up to compaction:
//   S1 activities, S2 row classes, S3 implied bounds (fused, one pass over the
//   CSR), S3'/S4 bound finalisation and fixing, S5 parallel rows.
//
// Load balance (Sec. 3.1, "length-based load balancing"): rows are grouped
// by length class.  Class c <= 5 gives each row a group of W = 2^c lanes of a
// warp (lane t walks entries t, t+W, ...; the group then reduces with an xor
// butterfly), class 6 (more than 4096 entries) splits the row into chunks of
// 4096 entries, one thread block each, whose partial results are combined in
// chunk order.  The order of every floating-point sum depends only on the
// row's own length.
//
// Bound tightening follows Sec. 3.1 in Jacobi form: activities and the
// acceptance tests read the bounds of the round start, accepted implied
// bounds are combined with atomicMin / atomicMax on an order-preserving
// integer encoding, which is exact and independent of the order of updates.
//
// FP64 is scarce on this GPU (about two DFMA per SM and clock), so every
// per-entry sign, finiteness and max(1,|x|) test runs on integer pipes, the
// activity sums are fused multiply-adds, and an implied bound is divided out
// only after an exact FMA sign test (x - thr*a) says it will be accepted.
#include <algorithm>
#include <cooperative_groups.h>

#include "lpp_launch.h"

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
__device__ __forceinline__ void touch_col(const Ctx &C, int32_t j) {
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
    C.lp_changed[lp] = 1;
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
    // (its lanes stay for the warp's queue steps).
    bool act = valid;
    if (valid && !C.rdirty[i]) {
        if (lane == 0) C.rkind[i] = RK_KEPT;
        act = false;
    }
    int32_t beg = 0, end = 0;
    if (act) {
        beg = C.A.ptr[i];
        end = C.A.ptr[i + 1];
    }
    const bool neg0 = end > beg ? is_neg(C.A.val[beg]) : false;
    double smin = 0.0, smax = 0.0;
    int nmin = 0, nmax = 0;
    unsigned long long h = 0;
#pragma unroll 4
    for (int32_t k = beg + lane; k < end; k += W) {  // unrolled: the bound gathers overlap (same order)
        const int32_t j = C.A.idx[k];
        const double a = C.A.val[k];
        const double2 b = C.lu[j];
        const bool neg = is_neg(a);
        const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
        if (is_fin(bmin)) smin = fma(a, bmin, smin);
        else nmin++;
        if (is_fin(bmax)) smax = fma(a, bmax, smax);
        else nmax++;
        h += entry_hash(j, neg != neg0);
    }
    smin = group_sum<W>(smin, mask);
    smax = group_sum<W>(smax, mask);
    nmin = group_sum<W>(nmin, mask);
    nmax = group_sum<W>(nmax, mask);
    h = group_sum<W>(h, mask);
    const int32_t len = end - beg;
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

__global__ void __launch_bounds__(kBlock, 4) k_prop_groups(Ctx C, GroupGrid g) {
    __shared__ double s_qx[kBlock / 32][kQueueCap], s_qa[kBlock / 32][kQueueCap];
    __shared__ int32_t s_qj[kBlock / 32][kQueueCap], s_qk[kBlock / 32][kQueueCap];
    __shared__ double s_ta[kBlock / 32][kQueueCap], s_ts[kBlock / 32][kQueueCap], s_tb[kBlock / 32][kQueueCap],
        s_to[kBlock / 32][kQueueCap];
    __shared__ int32_t s_tj[kBlock / 32][kQueueCap], s_tf[kBlock / 32][kQueueCap];
    const int warp = threadIdx.x >> 5;
    CandQueue q{s_qx[warp], s_qa[warp], s_qj[warp], s_qk[warp], 0};
    TestQueue tq{s_ta[warp], s_ts[warp], s_tb[warp], s_to[warp], s_tj[warp], s_tf[warp], 0};
    const int c = grid_class(g, blockIdx.x);
    const int32_t lb = blockIdx.x - g.blk_start[c];
    int32_t removed = 0, evaluated = 0, tested = 0;
    const int W = prop_lanes(c);
    const int32_t pos = C.A.cls_start[c] + lb * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    switch (c) {
        case 0:
        case 1:
        case 2: prop_group<1>(C, i, valid, removed, evaluated, tested, q, tq); break;
        case 3: prop_group<8>(C, i, valid, removed, evaluated, tested, q, tq); break;
        case 4: prop_group<16>(C, i, valid, removed, evaluated, tested, q, tq); break;
        default: prop_group<32>(C, i, valid, removed, evaluated, tested, q, tq); break;
    }
    tq_flush(C, tq, q);
    cq_flush(C, q);
    block_add(removed, &C.st->rows_removed);
    block_add(evaluated, &C.st->nnz_eval);
    block_add(tested, &C.st->sides_tested);
}

// fixed-order block reduction (warp butterflies, then warps in order)
template <typename T>
__device__ __forceinline__ T block_reduce_ordered(T v, T *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; w++) t += s_w[w];
    __syncthreads();
    return t;  // thread 0
}

// ------------------------------------------------------------ long rows
__global__ void __launch_bounds__(kBlock) k_prop_long_partial(Ctx C, unsigned long long *ch_hash) {
    __shared__ double s_d[kBlock / 32];
    __shared__ int s_i[kBlock / 32];
    __shared__ unsigned long long s_h[kBlock / 32];
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (!C.rdirty[ch.seg]) return;  // block-uniform
    const bool neg0 = is_neg(C.A.val[C.A.ptr[ch.seg]]);
    double smin = 0.0, smax = 0.0;
    int nmin = 0, nmax = 0;
    unsigned long long h = 0;
#pragma unroll 4
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) {
        const int32_t j = __ldcs(C.A.idx + k);  // streamed once: evict first, keep the bounds cached
        const double a = __ldcs(C.A.val + k);
        const double2 b = C.lu[j];
        const bool neg = is_neg(a);
        const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
        if (is_fin(bmin)) smin = fma(a, bmin, smin);
        else nmin++;
        if (is_fin(bmax)) smax = fma(a, bmax, smax);
        else nmax++;
        h += entry_hash(j, neg != neg0);
    }
    smin = block_reduce_ordered(smin, s_d);
    smax = block_reduce_ordered(smax, s_d);
    nmin = block_reduce_ordered(nmin, s_i);
    nmax = block_reduce_ordered(nmax, s_i);
    h = block_reduce_ordered(h, s_h);
    if (threadIdx.x == 0) {
        C.ch_act[blockIdx.x] = make_double2(smin, smax);
        C.ch_ninf[blockIdx.x] = make_int2(nmin, nmax);
        ch_hash[blockIdx.x] = h;
    }
}

// one warp per long row: the chunk partials, lane-strided then a butterfly
__global__ void __launch_bounds__(kBlock) k_prop_long_combine(Ctx C, const unsigned long long *ch_hash) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    int32_t removed = 0, evaluated = 0;
    if (t < nlong) {  // the same t in the whole warp
        const int32_t i = C.A.order[C.A.cls_start[6] + t];
        if (!C.rdirty[i]) {
            if (lane == 0) {
                C.rkind[i] = RK_KEPT;
                C.lneed[t] = 0;
            }
        } else {
            double smin = 0.0, smax = 0.0;
            int nmin = 0, nmax = 0;
            unsigned long long h = 0;
            for (int32_t q = C.A.lfirst[t] + lane; q < C.A.lfirst[t + 1]; q += 32) {
                const double2 a = C.ch_act[q];
                const int2 c = C.ch_ninf[q];
                smin += a.x;
                smax += a.y;
                nmin += c.x;
                nmax += c.y;
                h += ch_hash[q];
            }
            smin = group_sum<32>(smin, 0xffffffffu);
            smax = group_sum<32>(smax, 0xffffffffu);
            nmin = group_sum<32>(nmin, 0xffffffffu);
            nmax = group_sum<32>(nmax, 0xffffffffu);
            h = group_sum<32>(h, 0xffffffffu);
            if (lane == 0) {
                const int32_t beg = C.A.ptr[i], len = C.A.ptr[i + 1] - beg;
                h += len_hash(len);
                const double Lv = C.L[i], Uv = C.U[i];
                uint8_t kind;
                double sa = 0.0;
                int32_t sj = -1;  // long rows are never singletons
                removed = finish_row(C, i, beg, len, Lv, Uv, smin, smax, nmin, nmax, h, kind, sa, sj);
                evaluated = len;
                C.lneed[t] = kind == RK_KEPT && ((is_fin(Uv) && nmin <= 1) || (is_fin(Lv) && nmax <= 1));
            }
        }
    }
    block_add(removed, &C.st->rows_removed);
    block_add(evaluated, &C.st->nnz_eval);
}

__global__ void __launch_bounds__(kBlock) k_prop_long_tighten(Ctx C) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (!C.lneed[ch.lidx]) return;
    const int32_t i = ch.seg;
    const double Lv = C.L[i], Uv = C.U[i];
    const double2 act = C.act[i];
    const int2 ni = C.ninf[i];
    const bool up_row = is_fin(Uv) && ni.x <= 1, lo_row = is_fin(Lv) && ni.y <= 1;
    const double dU = Uv - act.x, dL = Lv - act.y;
    int32_t tested = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock)
        tighten_entry(C, C.A.idx[k], C.A.val[k], up_row, lo_row, dU, dL, ni.x, ni.y, tested);
    block_add(tested, &C.st->sides_tested);  // the whole block returned above or reaches here
}

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
            if (nl != b.x || nu != b.y) {
                C.lu[j] = make_double2(nl, nu);
                changed++;
                chg = 1;
                C.lp_changed[lp] = 1;
            }
            if (nl == nu) {
                kind = CK_FIXED;
                fixed++;
                C.fixv[j] = nl;
                const int32_t o = C.cmap[j];
                C.rec_ck[o] = CK_FIXED;
                C.rec_cr[o] = lp_round(C, lp);
                C.rec_cv[o] = nl;
                C.lp_changed[lp] = 1;
            }
        }
    }
    C.ckind[j] = kind;
    C.cchg[j] = chg;
    C.ctouch[j] = 0u;
    if (chg) {
        const int32_t len = C.T.ptr[j + 1] - C.T.ptr[j];
        if (len < kLongMin) coalesced_append(j, C.cl_cnt, C.cl_list);
        chg_nnz += len;
    }
}

// every column (some LP in its first round)
__global__ void __launch_bounds__(kBlock) k_colfin(Ctx C) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t changed = 0, fixed = 0, chg_nnz = 0;
    if (j < C.n) colfin_one(C, j, true, changed, fixed, chg_nnz);
    block_add(changed, &C.st->bounds_changed);
    block_add(fixed, &C.st->cols_fixed);
    block_add(chg_nnz, C.cl_nnz);
}

// the columns that received a candidate (the others keep their bounds; their
// kind and change flag were reset at the start of the round)
__global__ void __launch_bounds__(kBlock) k_colfin_list(Ctx C) {
    const int32_t cnt = *C.tl_cnt;
    int32_t changed = 0, fixed = 0, chg_nnz = 0;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
        colfin_one(C, C.tl_list[t], false, changed, fixed, chg_nnz);
    block_add(changed, &C.st->bounds_changed);
    block_add(fixed, &C.st->cols_fixed);
    block_add(chg_nnz, C.cl_nnz);
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

// first pass: rows kept by S2 with >= 2 entries take part
__global__ void __launch_bounds__(kBlock) k_s5_insert(Ctx C) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t part = 0;
    if (i < C.m) {
        int32_t slot = -1;
        if (C.rkind[i] == RK_KEPT && C.A.ptr[i + 1] - C.A.ptr[i] >= 2) slot = s5_insert_row(C, i, (uint32_t)C.tcap);
        C.rslot[i] = slot;
        C.rwork[i] = slot >= 0 ? 1 : 0;
        part = slot >= 0;
    }
    block_add(part, &C.st->participants);
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
    C.lp_changed[lp] = 1;
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

__global__ void __launch_bounds__(kBlock) k_s5_match_groups(Ctx C, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int32_t lb = blockIdx.x - g.blk_start[c];
    int32_t removed = 0, unmatched = 0;
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + lb * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    bool left;
    switch (c) {
        case 0: left = match_group<1>(C, i, valid, removed, unmatched); break;
        case 1: left = match_group<2>(C, i, valid, removed, unmatched); break;
        case 2: left = match_group<4>(C, i, valid, removed, unmatched); break;
        case 3: left = match_group<8>(C, i, valid, removed, unmatched); break;
        case 4: left = match_group<16>(C, i, valid, removed, unmatched); break;
        default: left = match_group<32>(C, i, valid, removed, unmatched); break;
    }
    block_add(removed, &C.st->rows_removed);
    block_add(unmatched, &C.st->unmatched);
    block_append(left, i, C.s5_out_cnt, C.s5_out);
}

// long rows: one block per row of class 6 (parallel long rows are rare)
__global__ void __launch_bounds__(kBlock) k_s5_match_long(Ctx C) {
    const int32_t t = blockIdx.x;
    const int32_t i = C.A.order[C.A.cls_start[6] + t];
    bool act = C.rwork[i] == 1;
    int32_t li = -1;
    if (act) {
        li = (int32_t)(uint32_t)(C.tlead[C.rslot[i]] & 0xffffffffULL);
        if (li == i) act = false;
    }
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
        for (int32_t k = threadIdx.x; k < len; k += kBlock) {
            const double ai = C.A.val[bi + k], al = C.A.val[bl + k];
            const double la = lam * al;
            if (!(C.A.idx[bi + k] == C.A.idx[bl + k] && fabs(ai - la) <= C.par_tol * fmax(fabs(ai), fabs(la))))
                ok = false;
        }
    }
    ok = __syncthreads_and(ok) != 0;
    int32_t removed = 0, unmatched = 0;
    if (threadIdx.x == 0) {
        if (act && ok) {
            s5_accept(C, i, li, lam);
            C.rwork[i] = 0;
            removed = 1;
        } else if (act) {
            C.rwork[i] = 2;
            unmatched = 1;
            C.s5_out[atomicAdd(C.s5_out_cnt, 1)] = i;
        } else {
            C.rwork[i] = 0;
        }
    }
    block_add(removed, &C.st->rows_removed);
    block_add(unmatched, &C.st->unmatched);
}

// Later passes run on the list of rows the previous pass left unmatched
// (count *cnt, at most the launch's grid): insert, match against the new
// leader (one warp per row; unmatched rows go to the next list), then clear
// the slots used so that the table is empty for the next pass.  The table
// capacity of a pass is the power of two >= 2 * count, at most C.tcap.
__device__ __forceinline__ uint32_t s5_tail_cap(const Ctx &C, int32_t n) {
    uint32_t cap = 1;
    while (cap < 2u * (uint32_t)n && cap < (uint32_t)C.tcap) cap <<= 1;
    return cap;
}

__global__ void __launch_bounds__(kBlock) k_s5_tail_insert(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t n = *cnt;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = list[t];
    C.rslot[i] = s5_insert_row(C, i, s5_tail_cap(C, n));
}

// one thread per listed row; rows longer than 32 entries are checked by the
// whole warp in turn
__global__ void __launch_bounds__(kBlock) k_s5_tail_match(Ctx C, const int32_t *list, const int32_t *cnt,
                                                         int32_t *out, int32_t *out_cnt) {
    const int32_t n = *cnt;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int32_t removed = 0;
    bool left = false, act = false, ok = false;
    int32_t i = -1, li = -1, bi = 0, bl = 0, len = 0;
    double lam = 0.0;
    if (t < n) {
        i = list[t];
        const int32_t sl = C.rslot[i];
        act = sl >= 0;
        if (act) {
            li = (int32_t)(uint32_t)(C.tlead[sl] & 0xffffffffULL);
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
    block_add(removed, &C.st->rows_removed);
    block_append(left, i, out_cnt, out);
}

__global__ void __launch_bounds__(kBlock) k_s5_tail_clear(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *cnt) return;
    const int32_t sl = C.rslot[list[t]];
    if (sl >= 0) {
        C.tkey[sl] = 0ULL;
        C.tlead[sl] = ~0ULL;
    }
}

// leaders take the followers' sides: L = max(L, merged), U = min(U, merged);
// crossing by more than the tolerance is infeasible, nearly equal sides snap
__global__ void __launch_bounds__(kBlock) k_s5_leader(Ctx C) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m || !C.hasf[i]) return;
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

// rows of a column whose bounds changed must be re-evaluated next round
// rows of the changed short columns need their activities next round: one
// thread per listed column; columns longer than 32 entries are walked by the
// whole warp in turn.  When the changed columns hold at least an eighth of the
// nonzeros, every row is marked instead (re-evaluating a row whose inputs did
// not change finds nothing new).
__global__ void __launch_bounds__(kBlock) k_mark_list(Ctx C, int64_t nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (8 * (int64_t)*C.cl_nnz >= nnz) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C.m; i += stride) C.rdnext[i] = 1;
        return;
    }
    const int32_t cnt = *C.cl_cnt;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += stride) {
        const int64_t t = base + lane;
        int32_t b = 0, e = 0;
        if (t < cnt) {
            const int32_t j = C.cl_list[t];
            b = C.T.ptr[j];
            e = C.T.ptr[j + 1];
        }
        if (e - b <= 32)
            for (int32_t k = b; k < e; k++) C.rdnext[C.T.idx[k]] = 1;
        unsigned todo = __ballot_sync(0xffffffffu, e - b > 32);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int32_t sb = __shfl_sync(0xffffffffu, b, src), se = __shfl_sync(0xffffffffu, e, src);
            for (int32_t k = sb + lane; k < se; k += 32) C.rdnext[C.T.idx[k]] = 1;
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_mark_long(Ctx C, int64_t nnz) {
    const Chunk ch = C.T.chunks[blockIdx.x];
    if (!C.cchg[ch.seg] || 8 * (int64_t)*C.cl_nnz >= nnz) return;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) C.rdnext[C.T.idx[k]] = 1;
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

}  // namespace

void launch_prop(const Ctx &C, cudaStream_t s) {
    GroupGrid g;  // blocks per class at prop_lanes(c) lanes per row
    int32_t acc = 0;
    for (int c = 0; c < 6; c++) {
        g.blk_start[c] = acc;
        const int32_t per = kBlock / prop_lanes(c);
        acc += (C.A.cls_start[c + 1] - C.A.cls_start[c] + per - 1) / per;
    }
    g.blk_start[6] = acc;
    if (g.blk_start[6] > 0) (k_prop_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    if (nlong > 0 && C.A.nchunks > 0) {
        (k_prop_long_partial<<<C.A.nchunks, kBlock, 0, s>>>(C, C.ch_hash), note_launch());
        (k_prop_long_combine<<<blocks_for((int64_t)nlong * 32, kBlock), kBlock, 0, s>>>(C, C.ch_hash), note_launch());
        (k_prop_long_tighten<<<C.A.nchunks, kBlock, 0, s>>>(C), note_launch());
    }
}

void launch_colfin(const Ctx &C, bool full, cudaStream_t s) {
    if (C.n <= 0) return;
    if (full) (k_colfin<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C), note_launch());
    else (k_colfin_list<<<std::min<unsigned>(blocks_for(C.n, kBlock), 8u * 152u), kBlock, 0, s>>>(C), note_launch());
}

void launch_mark_dirty(const Ctx &C, int64_t nnz, cudaStream_t s) {
    if (C.n <= 0) return;
    (k_mark_list<<<std::min<unsigned>(blocks_for(std::max(C.n, C.m), kBlock), 8u * 152u), kBlock, 0, s>>>(C, nnz),
     note_launch());
    if (C.T.cls_start[7] > C.T.cls_start[6] && C.T.nchunks > 0) (k_mark_long<<<C.T.nchunks, kBlock, 0, s>>>(C, nnz), note_launch());
}

void launch_s5_pass(const Ctx &C, cudaStream_t s) {
    if (C.m == 0) return;
    (k_s5_insert<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C), note_launch());
    const GroupGrid g = group_grid(C.A);
    if (g.blk_start[6] > 0) (k_s5_match_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    if (nlong > 0) (k_s5_match_long<<<nlong, kBlock, 0, s>>>(C), note_launch());
}

void launch_s5_tail(const Ctx &C, const int32_t *list, const int32_t *cnt, int32_t *out, int32_t *out_cnt,
                    int32_t max_rows, cudaStream_t s) {
    if (max_rows <= 0) return;
    (k_s5_tail_insert<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
    (k_s5_tail_match<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt, out, out_cnt), note_launch());
    (k_s5_tail_clear<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
}

void launch_s5_leader(const Ctx &C, cudaStream_t s) {
    if (C.m > 0) (k_s5_leader<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C), note_launch());
}

}  // namespace lpp
