// k_batch.cu -- batched presolve of many small LPs by one persistent kernel.
//
// Every thread block takes LPs from a queue (largest first) and runs the
// whole presolve loop of one LP at a time on the device: S1-S3 per row,
// S3'/S4 per column, S5 with all its leader passes, S6 and the compaction
// of the LP's CSR and CSC, round after round until the LP's round changes
// nothing, a verdict is reached or max_rounds have run.  No host round trip
// happens between rounds, and the LPs need no grid-wide synchronisation: each
// block owns the index ranges of its LP in every array of the arena (rows
// [row_off, row_off + m), columns [col_off, col_off + n), entries
// [nnz_off, nnz_off + nnz)) and compacts inside them.
//
// The per-row and per-column work is the one the round kernels launch over a
// whole arena (round_dev.cuh, compact_dev.cuh), with the same lanes per row
// (its length class), so an LP's records, maps and reduced LP are the same
// bits as from lpp_presolve alone.  Rows and columns of more than 4096
// entries are left to the per-round launches (the caller checks).
#include <algorithm>

#include "../../include/lpp.h"
#include "compact_dev.cuh"
#include "lpp_launch.h"
#include "round_dev.cuh"

namespace lpp {

namespace {

// ---------------------------------------------------------------- helpers
// Two exclusive scans of a[0, cnt) and b[0, cnt) by one block, into oa and
// ob (in place allowed): each thread sums a contiguous run of the input, the
// run totals are scanned across the block, then each thread writes its run.
// Returns both totals (every thread).  s_w: 2 (NT / 32) + 2 ints.
template <int NT>
__device__ int2 bscan2(const int32_t *a, const int32_t *b, int32_t *oa, int32_t *ob, int32_t cnt, int32_t *s_w) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t per = (cnt + NT - 1) / NT;
    const int32_t lo = min(cnt, (int32_t)threadIdx.x * per), hi = min(cnt, lo + per);
    int32_t sa = 0, sb = 0;
    for (int32_t t = lo; t < hi; t++) {
        sa += a[t];
        sb += b[t];
    }
    int32_t xa = sa, xb = sb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) {
            xa += ya;
            xb += yb;
        }
    }
    if (lane == 31) {
        s_w[warp] = xa;
        s_w[NW + warp] = xb;
    }
    __syncthreads();
    if (warp == 0) {
        int32_t wa = lane < NW ? s_w[lane] : 0, wb = lane < NW ? s_w[NW + lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t ya = __shfl_up_sync(0xffffffffu, wa, o), yb = __shfl_up_sync(0xffffffffu, wb, o);
            if (lane >= o) {
                wa += ya;
                wb += yb;
            }
        }
        if (lane < NW) {
            s_w[lane] = wa;
            s_w[NW + lane] = wb;
        }
    }
    __syncthreads();
    int32_t ca = (warp > 0 ? s_w[warp - 1] : 0) + xa - sa, cb = (warp > 0 ? s_w[NW + warp - 1] : 0) + xb - sb;
    for (int32_t t = lo; t < hi; t++) {
        const int32_t va = a[t], vb = b[t];
        oa[t] = ca;
        ob[t] = cb;
        ca += va;
        cb += vb;
    }
    const int2 tot = make_int2(s_w[NW - 1], s_w[2 * NW - 1]);
    __syncthreads();
    return tot;
}

// one block-wide sum of an int (every thread gets it)
template <int NT>
__device__ int32_t bsum(int32_t v, int32_t *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    int32_t t = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) t += s_w[w];
    __syncthreads();
    return t;
}

// shared state of a block: the LP's context and its sizes
struct BlockState {
    Ctx C;
    CompactCtx K;
    int32_t cls[8], fill[8];  // class starts of the row order, fill cursors
    int32_t k, cur, m, n, nnz, round;
    int32_t n1, n2;           // S5 list sizes
    int32_t w[34];            // scan / sum scratch
    int32_t act_buf, act_m;
};

__device__ void set_ctx(BlockState &S, const FusedArgs &F, const FusedLP &P) {
    const int k = S.k, b = S.cur;
    Ctx &C = S.C;
    C = F.base;
    C.A.ptr = F.frp[b] + k;
    C.A.idx = F.ci[b];
    C.A.val = F.rv[b];
    C.T.ptr = F.ftp[b] + k;
    C.T.idx = F.ti[b];
    C.T.val = F.tv[b];
    C.A.cnt = S.m;
    C.T.cnt = S.n;
    C.m = S.m;
    C.n = S.n;
    C.nlp = 1;
    C.round = S.round;
    C.list_touched = S.round > 1 ? 1 : 0;  // round 1's S3' checks every column
    C.L = F.L[b];
    C.U = F.U[b];
    C.rmap = F.rmap[b];
    C.lp_row = nullptr;
    C.act = F.act[b];
    C.ninf = F.ninf[b];
    C.hrow = F.hrow[b];
    C.rdirty = F.rdirty[b];
    C.lu = F.lu[b];
    C.c = F.c[b];
    C.cmap = F.cmap[b];
    C.lp_col = nullptr;
    C.tl_list = F.base.tl_list + P.col_off;
    C.tl_cnt = F.cnt + 4 * k;
    C.cl_list = F.base.cl_list + P.col_off;
    C.cl_cnt = F.cnt + 4 * k + 1;
    C.cl_nnz = F.cnt + 4 * k + 2;
    C.tkey = F.tkey + P.tab_off;
    C.tlead = F.tlead + P.tab_off;
    C.tcap = P.tcap;
    C.lp_round0 = nullptr;
    C.verdict = F.base.verdict + V_SLOTS * k;
    C.lp_changed = F.base.lp_changed + k;
    C.st = F.st + k;
    CompactCtx &K = S.K;
    K = F.K;
    K.lp_dead = F.dead + k;
    K.offset = F.K.offset + k;
}

// ------------------------------------------------------------- the kernel
template <int NT>
__global__ void __launch_bounds__(NT) k_batch_fused(FusedArgs F) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ BlockState S;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // per-warp candidate and test queues (the layout k_prop_groups uses)
    double *qd = reinterpret_cast<double *>(s_dyn);
    int32_t *qi = reinterpret_cast<int32_t *>(qd + 6 * NW * kQueueCap);
    CandQueue q{qd + (0 * NW + warp) * kQueueCap, qd + (1 * NW + warp) * kQueueCap,
                qi + (0 * NW + warp) * kQueueCap, qi + (1 * NW + warp) * kQueueCap, 0};
    TestQueue tq{qd + (2 * NW + warp) * kQueueCap, qd + (3 * NW + warp) * kQueueCap,
                 qd + (4 * NW + warp) * kQueueCap, qd + (5 * NW + warp) * kQueueCap,
                 qi + (2 * NW + warp) * kQueueCap, qi + (3 * NW + warp) * kQueueCap, 0};
    while (true) {
        if (tid == 0) {
            const int32_t t = atomicAdd(F.next, 1);
            S.k = t < F.count ? F.queue[t] : -1;
        }
        __syncthreads();
        if (S.k < 0) break;
        const int32_t k = S.k;
        const FusedLP P = F.lps[k];
        const int32_t r0 = P.row_off, c0 = P.col_off, z0 = P.nnz_off;
        // the LP's pointers into buffer 0
        for (int32_t t = tid; t <= P.m; t += NT) F.frp[0][k + r0 + t] = F.rp0[r0 + t];
        for (int32_t t = tid; t <= P.n; t += NT) F.ftp[0][k + c0 + t] = F.tp0[c0 + t];
        if (tid == 0) {
            S.cur = 0;
            S.m = P.m;
            S.n = P.n;
            S.nnz = P.nnz;
            S.act_buf = 0;
            S.act_m = P.m;
        }
        int32_t status = LPP_OK, where = LPP_WHERE_NONE, vindex = -1, vround = 0, rounds = 0;
        long long s5_left = 0;
        bool s5_clean = false;  // the last S5 resolved every group and no row changed since
        __syncthreads();
        for (int32_t r = 1; r <= F.max_rounds; r++) {
            if (tid == 0) {
                S.round = r;
                set_ctx(S, F, P);
                *S.C.st = DevStatus{};
                *S.C.lp_changed = 0;
                S.C.tl_cnt[0] = 0;
                S.C.cl_cnt[0] = 0;
                S.C.cl_nnz[0] = 0;
                S.act_buf = S.cur;
                S.act_m = S.m;
                for (int c = 0; c < 8; c++) S.cls[c] = 0;
            }
            __syncthreads();
            const Ctx &C = S.C;
            const int32_t m = S.m, n = S.n, nnz = S.nnz;
            if (r > 1)
                for (int32_t j = c0 + tid; j < c0 + n; j += NT) {
                    C.ckind[j] = CK_KEPT;
                    C.cchg[j] = 0;
                }
            for (int32_t i = r0 + tid; i < r0 + m; i += NT) C.rdnext[i] = 0;
            // rows by length class (one shared atomic per class and warp step)
            for (int32_t i0 = r0 + warp * 32; i0 < r0 + m; i0 += NT) {
                const int32_t i = i0 + lane;
                const int c = i < r0 + m ? seg_class(C.A.ptr[i + 1] - C.A.ptr[i]) : 7;
                const unsigned peers = __match_any_sync(0xffffffffu, c);
                if (c < 7 && lane == __ffs(peers) - 1) atomicAdd(&S.cls[c], __popc(peers));
            }
            __syncthreads();
            if (tid == 0) {
                int32_t a = 0;
                for (int c = 0; c < 8; c++) {
                    const int32_t v = S.cls[c];
                    S.cls[c] = a;
                    S.fill[c] = a;
                    a += v;
                }
            }
            __syncthreads();
            for (int32_t i0 = r0 + warp * 32; i0 < r0 + m; i0 += NT) {
                const int32_t i = i0 + lane;
                const int c = i < r0 + m ? seg_class(C.A.ptr[i + 1] - C.A.ptr[i]) : 7;
                const unsigned peers = __match_any_sync(0xffffffffu, c);
                const int first = __ffs(peers) - 1;
                int32_t base = 0;
                if (c < 7 && lane == first) base = atomicAdd(&S.fill[c], __popc(peers));
                base = __shfl_sync(0xffffffffu, base, first);
                if (c < 7) F.order[r0 + base + __popc(peers & ((1u << lane) - 1u))] = i;
            }
            __syncthreads();
            const int32_t *ord = F.order + r0;

            // S1 + S2 + S3: W lanes per row (prop_lanes of its class)
            int32_t rem = 0, evaluated = 0, tested = 0;
            for (int c = 0; c < 6; c++) {
                const int W = prop_lanes(c), per = 32 / W;
                const int32_t b0 = S.cls[c], cnt = S.cls[c + 1] - b0;
                const int32_t packets = (cnt + per - 1) / per;
                for (int32_t p = warp; p < packets; p += NW) {
                    const int32_t pos = p * per + lane / W;
                    const bool valid = pos < cnt;
                    const int32_t i = valid ? ord[b0 + pos] : 0;
                    switch (W) {
                        case 1: prop_group<1>(C, i, valid, rem, evaluated, tested, q, tq); break;
                        case 8: prop_group<8>(C, i, valid, rem, evaluated, tested, q, tq); break;
                        case 16: prop_group<16>(C, i, valid, rem, evaluated, tested, q, tq); break;
                        default: prop_group<32>(C, i, valid, rem, evaluated, tested, q, tq); break;
                    }
                }
            }
            tq_flush(C, tq, q);
            cq_flush(C, q);
            int32_t removed = bsum<NT>(rem, S.w);
            rem = 0;
            // S3' + S4: every column in round 1, else the columns that received a candidate
            int32_t changed = 0, fixed = 0, chg_nnz = 0;
            if (r == 1) {
                for (int32_t j = c0 + tid; j < c0 + n; j += NT) colfin_one(C, j, true, changed, fixed, chg_nnz);
            } else {
                const int32_t tc = C.tl_cnt[0];
                for (int32_t t = tid; t < tc; t += NT) colfin_one(C, C.tl_list[t], false, changed, fixed, chg_nnz);
            }
            changed = bsum<NT>(changed, S.w);
            fixed = bsum<NT>(fixed, S.w);
            chg_nnz = bsum<NT>(chg_nnz, S.w);
            // rows of columns whose bounds changed are evaluated next round
            // (every row when those columns hold an eighth of the entries)
            if (8 * (int64_t)chg_nnz >= nnz) {
                for (int32_t i = r0 + tid; i < r0 + m; i += NT) C.rdnext[i] = 1;
            } else {
                const int32_t cc = C.cl_cnt[0];
                for (int32_t t = tid; t < cc; t += NT) {
                    const int32_t j = C.cl_list[t];
                    for (int32_t e = C.T.ptr[j]; e < C.T.ptr[j + 1]; e++) C.rdnext[C.T.idx[e]] = 1;
                }
            }

            // S5, first pass: rows S2 kept with >= 2 entries, leaders elected in
            // the LP's table, then every row against its leader (class width W).
            // Skipped when the last S5 resolved every key group and no row lost
            // an entry since (it would remove nothing).
            const bool run_s5 = r == 1 || !s5_clean;
            for (int32_t i = r0 + tid; i < r0 + m && run_s5; i += NT) {
                int32_t slot = -1;
                if (C.rkind[i] == RK_KEPT && C.A.ptr[i + 1] - C.A.ptr[i] >= 2) slot = s5_insert_row(C, i, (uint32_t)P.tcap);
                C.rslot[i] = slot;
                C.rwork[i] = slot >= 0 ? 1 : 0;
            }
            if (tid == 0) {
                S.n1 = 0;
                S.n2 = 0;
            }
            __syncthreads();
            int32_t unmatched = 0;
            for (int c = 0; c < 6 && run_s5; c++) {
                const int W = 1 << c, per = 32 / W;
                const int32_t b0 = S.cls[c], cnt = S.cls[c + 1] - b0;
                const int32_t packets = (cnt + per - 1) / per;
                for (int32_t p = warp; p < packets; p += NW) {
                    const int32_t pos = p * per + lane / W;
                    const bool valid = pos < cnt;
                    const int32_t i = valid ? ord[b0 + pos] : 0;
                    bool left;
                    switch (c) {
                        case 0: left = match_group<1>(C, i, valid, rem, unmatched); break;
                        case 1: left = match_group<2>(C, i, valid, rem, unmatched); break;
                        case 2: left = match_group<4>(C, i, valid, rem, unmatched); break;
                        case 3: left = match_group<8>(C, i, valid, rem, unmatched); break;
                        case 4: left = match_group<16>(C, i, valid, rem, unmatched); break;
                        default: left = match_group<32>(C, i, valid, rem, unmatched); break;
                    }
                    if (left) F.list[0][r0 + atomicAdd(&S.n1, 1)] = i;
                }
            }
            __syncthreads();
            // the table empty again
            for (int32_t i = r0 + tid; i < r0 + m && run_s5; i += NT) {
                const int32_t sl = C.rslot[i];
                if (sl >= 0) {
                    C.tkey[sl] = 0ULL;
                    C.tlead[sl] = ~0ULL;
                }
            }
            __syncthreads();
            // later passes on the rows left unmatched, at most par_max_iter in all
            int32_t ncur = S.n1, from = 0;
            for (int32_t pass = 1; pass < F.par_max_iter && ncur > 0; pass++) {
                const int32_t *lst = F.list[from] + r0;
                int32_t *nxt = F.list[from ^ 1] + r0;
                const uint32_t cap = s5_tail_cap(C, ncur);
                for (int32_t t = tid; t < ncur; t += NT) C.rslot[lst[t]] = s5_insert_row(C, lst[t], cap);
                if (tid == 0) S.n2 = 0;
                __syncthreads();
                for (int32_t tb = warp * 32; tb < ncur; tb += NT) {
                    int32_t rm, i;
                    bool left;
                    s5_tail_match_one(C, lst, ncur, tb + lane, rm, left, i);
                    rem += rm;
                    if (left) nxt[atomicAdd(&S.n2, 1)] = i;
                }
                __syncthreads();
                for (int32_t t = tid; t < ncur; t += NT) {
                    const int32_t sl = C.rslot[lst[t]];
                    if (sl >= 0) {
                        C.tkey[sl] = 0ULL;
                        C.tlead[sl] = ~0ULL;
                    }
                }
                __syncthreads();
                ncur = S.n2;
                from ^= 1;
            }
            // rows still unmatched at the pass cap (all passes ran)
            if (ncur > 0) s5_left += ncur;
            if (run_s5) s5_clean = ncur == 0;
            for (int32_t i = r0 + tid; i < r0 + m; i += NT)
                if (C.hasf[i]) s5_leader_one(C, i);
            removed += bsum<NT>(rem, S.w);
            __syncthreads();

            // verdict of this round's S2, S3', S5 (first in step order)
            int v = 0;
            while (v < V_SLOTS && C.verdict[v] == kNone) v++;
            const bool dead = v < V_SLOTS;
            const bool structural = r == 1 || removed > 0 || fixed > 0 || dead;
            if (structural && !dead) {
                const CompactCtx &K = S.K;
                // S6 inputs: entries of each column in kept rows, locks
                for (int32_t j = c0 + tid; j < c0 + n; j += NT) {
                    int32_t cnt = 0, lk = 0;
                    for (int32_t e = C.T.ptr[j]; e < C.T.ptr[j + 1]; e++) {
                        const int32_t i = C.T.idx[e];
                        cnt += C.rkind[i] == RK_KEPT;
                        if (C.dualfix) lk |= entry_locks(C, i, C.T.val[e]);
                    }
                    K.c_len[j] = cnt;
                    if (C.dualfix) K.c_lock[j] = lk;
                }
                __syncthreads();
                int32_t sfix = 0;
                for (int32_t j = c0 + tid; j < c0 + n; j += NT) sfix += colkeep_one(C, K, j);
                fixed += bsum<NT>(sfix, S.w);
                // per row: kept entries and the side shift (class width W)
                for (int c = 0; c < 6; c++) {
                    const int W = 1 << c, per = 32 / W;
                    const int32_t b0 = S.cls[c], cnt = S.cls[c + 1] - b0;
                    const int32_t packets = (cnt + per - 1) / per;
                    for (int32_t p = warp; p < packets; p += NW) {
                        const int32_t pos = p * per + lane / W;
                        const bool valid = pos < cnt;
                        const int32_t i = valid ? ord[b0 + pos] : 0;
                        const bool keep = valid && C.rkind[i] == RK_KEPT;
                        switch (c) {
                            case 0: csr_count_row<1>(C, K, i, valid, keep); break;
                            case 1: csr_count_row<2>(C, K, i, valid, keep); break;
                            case 2: csr_count_row<4>(C, K, i, valid, keep); break;
                            case 3: csr_count_row<8>(C, K, i, valid, keep); break;
                            case 4: csr_count_row<16>(C, K, i, valid, keep); break;
                            default: csr_count_row<32>(C, K, i, valid, keep); break;
                        }
                    }
                }
                __syncthreads();
                // objective constant: the LP's columns lane-strided, then a butterfly
                if (warp == 0) {
                    double s = 0.0;
                    for (int32_t j = c0 + lane; j < c0 + n; j += 32) s += K.contrib[j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) K.offset[0] += s;
                }
                // new indices and offsets
                const int2 rt = bscan2<NT>(K.r_keep + r0, K.r_len + r0, K.r_pos + r0, K.r_off + r0, m, S.w);
                const int2 ct = bscan2<NT>(K.c_keep + c0, K.c_len + c0, K.c_pos + c0, K.c_off + c0, n, S.w);
                const int32_t m2 = rt.x, z2 = rt.y, n2 = ct.x, z2t = ct.y;
                const int nx = S.cur ^ 1;
                int32_t *rp2 = F.frp[nx] + k, *tp2 = F.ftp[nx] + k;
                for (int32_t i = r0 + tid; i < r0 + m; i += NT) {
                    const bool kp = K.r_keep[i] != 0;
                    const int32_t p = r0 + K.r_pos[i];
                    K.r_new[i] = kp ? p : -1;
                    if (!kp) continue;
                    const double sh = K.shift[i], Lv = C.L[i], Uv = C.U[i];
                    F.L[nx][p] = is_fin(Lv) ? Lv - sh : Lv;
                    F.U[nx][p] = is_fin(Uv) ? Uv - sh : Uv;
                    F.rmap[nx][p] = C.rmap[i];
                    rp2[p] = z0 + K.r_off[i];
                    // a row that lost entries changed: evaluate it next round;
                    // an unchanged row's S5 key is taken again when columns
                    // were dropped (it hashes the renumbered column indices)
                    const bool lost = K.r_len[i] != C.A.ptr[i + 1] - C.A.ptr[i];
                    F.rdirty[nx][p] = (C.rdnext[i] | lost) ? 1 : (n2 != n ? 2 : 0);
                    F.act[nx][p] = C.act[i];
                    F.ninf[nx][p] = C.ninf[i];
                    F.hrow[nx][p] = C.hrow[i];
                }
                for (int32_t j = c0 + tid; j < c0 + n; j += NT) {
                    const bool kp = K.c_keep[j] != 0;
                    const int32_t p = c0 + K.c_pos[j];
                    K.c_new[j] = kp ? p : -1;
                    if (!kp) continue;
                    F.lu[nx][p] = C.lu[j];
                    F.c[nx][p] = C.c[j];
                    F.cmap[nx][p] = C.cmap[j];
                    tp2[p] = z0 + K.c_off[j];
                }
                if (tid == 0) {
                    rp2[r0 + m2] = z0 + z2;
                    tp2[c0 + n2] = z0 + z2t;
                }
                __syncthreads();
                // entries: a kept row's entries in kept columns, renumbered, in
                // order (a thread per row up to 32 entries, else its warp)
                for (int pass2 = 0; pass2 < 2; pass2++) {
                    const bool rows = pass2 == 0;
                    const int32_t cnt = rows ? m : n, base = rows ? r0 : c0;
                    const int32_t *ptr = rows ? C.A.ptr : C.T.ptr;
                    const int32_t *idx = rows ? C.A.idx : C.T.idx;
                    const double *val = rows ? C.A.val : C.T.val;
                    const int32_t *keep = rows ? K.r_keep : K.c_keep;
                    const int32_t *off = rows ? K.r_off : K.c_off;
                    const int32_t *nw = rows ? K.c_new : K.r_new;
                    int32_t *oi = rows ? F.ci[nx] : F.ti[nx];
                    double *ov = rows ? F.rv[nx] : F.tv[nx];
                    for (int32_t s0 = base + warp * 32; s0 < base + cnt; s0 += NT) {
                        const int32_t sg = s0 + lane;
                        const bool own = sg < base + cnt && keep[sg];
                        int32_t b = 0, e = 0, o = 0;
                        if (own) {
                            b = ptr[sg];
                            e = ptr[sg + 1];
                            o = z0 + off[sg];
                        }
                        if (own && e - b <= 32)
                            for (int32_t x = b; x < e; x++) {
                                const int32_t ni = nw[idx[x]];
                                if (ni >= 0) {
                                    oi[o] = ni;
                                    ov[o] = val[x];
                                    o++;
                                }
                            }
                        unsigned todo = __ballot_sync(0xffffffffu, own && e - b > 32);
                        while (todo) {
                            const int src = __ffs(todo) - 1;
                            todo &= todo - 1u;
                            const int32_t sb = __shfl_sync(0xffffffffu, b, src), se = __shfl_sync(0xffffffffu, e, src);
                            int32_t so = __shfl_sync(0xffffffffu, o, src);
                            for (int32_t x0 = sb; x0 < se; x0 += 32) {
                                const int32_t x = x0 + lane;
                                const int32_t ni = x < se ? nw[idx[x]] : -1;
                                const unsigned bal = __ballot_sync(0xffffffffu, ni >= 0);
                                if (ni >= 0) {
                                    const int32_t at = so + __popc(bal & ((1u << lane) - 1u));
                                    oi[at] = ni;
                                    ov[at] = val[x];
                                }
                                so += __popc(bal);
                            }
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    S.cur = nx;
                    S.m = m2;
                    S.n = n2;
                    S.nnz = z2;
                }
            } else if (dead) {
                if (tid == 0) {
                    S.m = 0;
                    S.n = 0;
                    S.nnz = 0;
                    S.K.lp_dead[0] = 1;
                }
            } else {  // same numbering: the flags gathered this round
                uint8_t *rd = F.rdirty[S.cur];
                for (int32_t i = r0 + tid; i < r0 + m; i += NT) rd[i] = C.rdnext[i];
            }
            if (fixed > 0) s5_clean = false;  // rows lost entries (S4 or S6 fixings)
            __syncthreads();
            // round end: counters, then the LP's verdict or convergence
            if (tid == 0) {
                int32_t *rs = F.rstat + 4 * ((int64_t)k * F.max_rounds + (r - 1));
                rs[0] = nnz;
                rs[1] = removed;
                rs[2] = fixed;
                rs[3] = changed;
            }
            rounds = r;
            int vv = 0;
            while (vv < V_SLOTS && C.verdict[vv] == kNone) vv++;
            if (vv < V_SLOTS) {
                status = vv == V_S6_COL ? LPP_UNBOUNDED : LPP_INFEASIBLE;
                where = (vv == V_S2_ROW || vv == V_S5_ROW) ? LPP_WHERE_ROW : LPP_WHERE_COL;
                vindex = C.verdict[vv];
                vround = r;
                break;
            }
            const bool chg = *C.lp_changed != 0;
            __syncthreads();
            if (!chg) break;
        }
        __syncthreads();
        // the LP's results: reduced LP (LP-local indices), final bounds and
        // maps, the activities of its last round, its verdict and counters
        {
            const int b = S.cur;
            const int32_t m = S.m, n = S.n, nnz = S.nnz;
            const int32_t *rp = F.frp[b] + k, *tp = F.ftp[b] + k;
            for (int32_t t = tid; t <= m; t += NT) F.o_rp[k + r0 + t] = m > 0 ? rp[r0 + t] - z0 : 0;
            for (int32_t t = tid; t <= n; t += NT) F.o_tp[k + c0 + t] = n > 0 ? tp[c0 + t] - z0 : 0;
            for (int32_t e = tid; e < nnz; e += NT) {
                F.o_ci[z0 + e] = F.ci[b][z0 + e] - c0;
                F.o_rv[z0 + e] = F.rv[b][z0 + e];
                F.o_ti[z0 + e] = F.ti[b][z0 + e] - r0;
                F.o_tv[z0 + e] = F.tv[b][z0 + e];
            }
            for (int32_t t = tid; t < m; t += NT) {
                F.o_L[r0 + t] = F.L[b][r0 + t];
                F.o_U[r0 + t] = F.U[b][r0 + t];
                F.o_rmap[r0 + t] = F.rmap[b][r0 + t] - r0;
            }
            for (int32_t t = tid; t < n; t += NT) {
                const double2 lu = F.lu[b][c0 + t];
                F.o_c[c0 + t] = F.c[b][c0 + t];
                F.o_lb[c0 + t] = lu.x;
                F.o_ub[c0 + t] = lu.y;
                F.o_lu[c0 + t] = lu;
                F.o_cmap[c0 + t] = F.cmap[b][c0 + t] - c0;
                F.o_fcmap[c0 + t] = F.cmap[b][c0 + t];
            }
            const int32_t am = S.act_m, ab = S.act_buf;
            for (int32_t t = tid; t < am; t += NT) {
                F.o_act[r0 + t] = F.act[ab][r0 + t];
                F.o_ninf[r0 + t] = F.ninf[ab][r0 + t];
                F.o_armap[r0 + t] = F.rmap[ab][r0 + t];
            }
            if (tid == 0) {
                FusedOut o;
                o.status = status;
                o.where = where;
                o.index = vindex;
                o.round = vround;
                o.rounds = rounds;
                o.m = m;
                o.n = n;
                o.nnz = nnz;
                o.act_m = am;
                o.pad = 0;
                o.s5_left = s5_left;
                F.out[k] = o;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t batch_fused_smem(int threads) { return (size_t)(threads / 32) * kQueueCap * (6 * sizeof(double) + 4 * sizeof(int32_t)); }

int batch_fused_blocks_per_sm(int threads) {
    int b = 0;
    cudaError_t e = cudaSuccess;
    if (threads == 512)
        cudaFuncSetAttribute(k_batch_fused<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_fused_smem(512));
    switch (threads) {
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fused<128>, 128, batch_fused_smem(128)); break;
        case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fused<256>, 256, batch_fused_smem(256)); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fused<512>, 512, batch_fused_smem(512)); break;
    }
    return e == cudaSuccess ? b : 0;
}

void launch_batch_fused(const FusedArgs &F, int threads, int blocks, cudaStream_t s) {
    const size_t smem = batch_fused_smem(threads);
    switch (threads) {
        case 128: (k_batch_fused<128><<<blocks, 128, smem, s>>>(F), note_launch()); break;
        case 256: (k_batch_fused<256><<<blocks, 256, smem, s>>>(F), note_launch()); break;
        default:
            cudaFuncSetAttribute(k_batch_fused<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            (k_batch_fused<512><<<blocks, 512, smem, s>>>(F), note_launch());
            break;
    }
}

}  // namespace lpp
