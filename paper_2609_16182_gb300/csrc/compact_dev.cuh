// compact_dev.cuh -- the per-column and per-row work of S6 and of the
// compaction counts (S7), shared by the compaction kernels (k_compact.cu)
// and the fused batch kernel (k_batch.cu).
#pragma once
#include "lpp_dev.cuh"

namespace lpp {

namespace {

// ------------------------------------------------- locks (dual fixing, S6)
// A kept row a_ij x_j + ... in [L_i, U_i] locks x_j downwards when a_ij > 0
// and L_i is finite or a_ij < 0 and U_i is finite, upwards in the mirrored
// cases: bit 1 = down, bit 2 = up, OR-combined over the column.
__device__ __forceinline__ int32_t entry_locks(const Ctx &C, int32_t i, double a) {
    if (C.rkind[i] != RK_KEPT) return 0;
    const int32_t fl = is_fin(C.L[i]), fu = is_fin(C.U[i]);
    return is_neg(a) ? (fu | (fl << 1)) : (fl | (fu << 1));
}

// S6 and the keep flag of column j (after the counts of its entries in kept
// rows, K.c_len, and with opts.dual_fixing its locks, K.c_lock): a column
// with no entry left, or no lock in the direction its cost prefers, is
// fixed at that bound (an infinite one is the UNBOUNDED verdict); K.contrib
// gets c_j v_j of a column that leaves with a value.  Returns 1 if S6 fixed it.
__device__ __forceinline__ int32_t colkeep_one(const Ctx &C, const CompactCtx &K, int32_t j) {
    int32_t fixed = 0;
    const int32_t lp = lp_of_col(C, j);
    const bool dead = K.lp_dead[lp];
    uint8_t kind = C.ckind[j];
    double contrib = 0.0;
    if (!dead && kind == CK_KEPT && C.dual && (K.c_len[j] == 0 || C.dualfix)) {
        // the bound the cost prefers, when no kept row locks the column in
        // that direction (an empty column has no locks)
        const int32_t lk = K.c_len[j] == 0 ? 0 : K.c_lock[j];
        const bool dl = lk & 1, ul = lk & 2;
        const double2 b = C.lu[j];
        const double cj = C.c[j];
        double v;
        bool fix;
        if (cj > 0.0) { fix = !dl; v = b.x; }
        else if (cj < 0.0) { fix = !ul; v = b.y; }
        else if (!dl && is_fin(b.x)) { fix = true; v = b.x; }
        else if (!ul && is_fin(b.y)) { fix = true; v = b.y; }
        else { fix = !dl && !ul; v = 0.0; }
        if (!fix) {
            // locked: kept
        } else if (!is_fin(v)) {
            atomicMin(&C.verdict[lp * V_SLOTS + V_S6_COL], C.cmap[j]);
        } else {
            kind = CK_EMPTY;
            C.ckind[j] = kind;
            C.fixv[j] = v;
            const int32_t o = C.cmap[j];
            C.rec_ck[o] = CK_EMPTY;
            C.rec_cr[o] = lp_round(C, lp);
            C.rec_cv[o] = v;
            mark_lp_changed(C, lp);
            fixed = 1;
        }
    }
    if (!dead && kind != CK_KEPT && kind != CK_PARALLEL) contrib = C.c[j] * C.fixv[j];  // merged: none
    const bool keep = !dead && kind == CK_KEPT;
    K.c_keep[j] = keep;
    if (!keep) K.c_len[j] = 0;
    K.contrib[j] = contrib;
    return fixed;
}

// Row i of W lanes (its length class): its entries left in kept columns
// (K.r_len) and the side shift sum_j a_ij v_j over its columns that leave
// with a value (K.shift: lane-strided fused multiply-adds, then the group's
// butterfly), if `keep`; K.r_keep.
template <int W>
__device__ __forceinline__ void csr_count_row(const Ctx &C, const CompactCtx &K, int32_t i, bool valid,
                                              bool keep) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    int32_t beg = 0, end = 0;
    if (keep) {
        beg = C.A.ptr[i];
        end = C.A.ptr[i + 1];
    }
    int32_t cnt = 0;
    double sh = 0.0;
    // four entries per lane and step: their indices, then their keep flags,
    // in flight together; the shift takes the entries in order
    for (int32_t k0 = beg + lane; k0 < end; k0 += 4 * W) {
        int32_t jq[4], kq[4];
#pragma unroll
        for (int q = 0; q < 4; q++) jq[q] = k0 + q * W < end ? C.A.idx[k0 + q * W] : 0;
#pragma unroll
        for (int q = 0; q < 4; q++) kq[q] = k0 + q * W < end ? K.c_keep[jq[q]] : 1;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (k0 + q * W >= end) break;
            if (kq[q]) cnt++;
            else sh = fma(C.A.val[k0 + q * W], C.fixv[jq[q]], sh);
        }
    }
    cnt = group_sum<W>(cnt, mask);
    sh = group_sum<W>(sh, mask);
    if (valid && lane == 0) {
        K.r_keep[i] = keep;
        K.r_len[i] = cnt;
        K.shift[i] = sh;
    }
}

}  // namespace

}  // namespace lpp
