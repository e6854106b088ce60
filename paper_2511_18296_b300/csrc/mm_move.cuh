// Move decoding and the exact integer feasibility test, shared by the
// evaluation and apply kernels.
//
// Precedence (Eq. 15): every arc p -> c needs x_p <= x_c.  With the packed
// lo/hi bounds of each block (lo = latest predecessor period, hi = earliest
// successor period), moving block b to t' keeps every arc at b iff
// lo_b <= t' <= hi_b, because only b's own period changes.  For a swap of b1
// and b2 the two bounds are checked independently; when b2 is itself a direct
// predecessor (successor) of b1 the bounds contain b2's old period, which is
// harmless (it equals the other side of the inequality), and the arc between
// them is checked in its new orientation: t1 <= t2 (t2 <= t1).
// Capacity (Eq. 16): every period a moved block leaves or enters must hold
// at most M_t tonnes afterwards.  Tonnages are integers, so the flag is exact.
#pragma once

#include "mm_internal.cuh"

namespace mm {

struct MoveView {
    int32_t b1, b2;        // b2 = -1 for a shift
    uint32_t t1, t2;       // b1 moves t1 -> t2; for a swap b2 moves t2 -> t1
    uint32_t m1, m2;       // masses (m2 = 0 for a shift)
    bool swap, valid, feasible, noop;
};

struct Topo {
    int32_t B, T, nx, ny, nz;
    const int32_t *pred_ptr, *pred_idx, *succ_ptr, *succ_idx;  // CSR when nx == 0
};

// Compact 4-byte move p = (b1 << 16) | code (needs B + T + 1 <= 65536):
// code < B swaps b1 with block `code`, code = 65535 - t shifts b1 to period t
// (0..T); any other code, or b1 >= B, is the bad move {-1, -1}.
__device__ __forceinline__ int2 unpack_move(uint32_t p, int32_t B, int32_t T) {
    const int32_t b1 = (int32_t)(p >> 16), code = (int32_t)(p & 0xffffu);
    if (b1 < B) {
        if (code < B) return make_int2(b1, code);
        if (code >= 65535 - T) return make_int2(b1, -(65535 - code) - 1);
    }
    return make_int2(-1, -1);
}

// Is a a direct predecessor of b?  (1-5 pattern or CSR)
__device__ __forceinline__ bool is_pred(const Topo &tp, int32_t a, int32_t b) {
    if (tp.nx > 0) {
        int32_t nxy = tp.nx * tp.ny;
        int32_t d = b - a;
        if (d < nxy - tp.nx || d > nxy + tp.nx) return false;  // cheap filter
        int32_t xb = b % tp.nx, yb = (b / tp.nx) % tp.ny, zb = b / nxy;
        int32_t xa = a % tp.nx, ya = (a / tp.nx) % tp.ny, za = a / nxy;
        if (za != zb - 1) return false;
        int32_t dx = xa - xb, dy = ya - yb;
        return (dx == 0 && (dy == 0 || dy == 1 || dy == -1)) || (dy == 0 && (dx == 1 || dx == -1));
    }
    for (int32_t k = tp.pred_ptr[b]; k < tp.pred_ptr[b + 1]; k++)
        if (tp.pred_idx[k] == a) return true;
    return false;
}

template <typename LoadBlk, typename LoadMass, typename Mined, typename Cap>
__device__ __forceinline__ MoveView decode_move(int2 mv, const Topo &tp, LoadBlk load_blk, LoadMass load_mass,
                                                Mined mined, Cap cap) {
    MoveView v;
    v.b1 = mv.x;
    v.swap = mv.y >= 0;
    v.b2 = v.swap ? mv.y : -1;
    int32_t tn = -mv.y - 1;
    v.valid = (mv.x >= 0) && (mv.x < tp.B) && (v.swap ? (mv.y < tp.B) : (tn >= 0 && tn <= tp.T));
    v.feasible = false;
    v.noop = true;
    v.t1 = v.t2 = 0;
    v.m1 = v.m2 = 0;
    if (!v.valid) return v;
    uint32_t w1 = load_blk(v.b1);
    v.t1 = blk_period(w1);
    v.m1 = load_mass(v.b1);
    bool ok;
    if (v.swap) {
        uint32_t w2 = load_blk(v.b2);
        v.t2 = blk_period(w2);
        v.m2 = load_mass(v.b2);
        v.noop = (v.b1 == v.b2) || (v.t1 == v.t2);
        ok = blk_lo(w1) <= v.t2 && v.t2 <= blk_hi(w1) && blk_lo(w2) <= v.t1 && v.t1 <= blk_hi(w2);
        if (ok && v.b1 != v.b2 && v.t1 != v.t2) {
            if (is_pred(tp, v.b2, v.b1)) ok = v.t1 <= v.t2;       // arc b2 -> b1 after the swap
            else if (is_pred(tp, v.b1, v.b2)) ok = v.t2 <= v.t1;  // arc b1 -> b2 after the swap
        }
        if (ok) {
            if (v.noop) {
                if (v.t1 < (uint32_t)tp.T) ok = (uint64_t)mined(v.t1) <= cap(v.t1);
            } else {
                if (v.t1 < (uint32_t)tp.T)
                    ok = (uint64_t)(mined(v.t1) - (int64_t)v.m1 + (int64_t)v.m2) <= cap(v.t1);
                if (ok && v.t2 < (uint32_t)tp.T)
                    ok = (uint64_t)(mined(v.t2) - (int64_t)v.m2 + (int64_t)v.m1) <= cap(v.t2);
            }
        }
    } else {
        v.t2 = (uint32_t)tn;
        v.noop = v.t1 == v.t2;
        ok = blk_lo(w1) <= v.t2 && v.t2 <= blk_hi(w1);
        if (ok) {
            if (v.noop) {
                if (v.t1 < (uint32_t)tp.T) ok = (uint64_t)mined(v.t1) <= cap(v.t1);
            } else {
                if (v.t1 < (uint32_t)tp.T) ok = (uint64_t)(mined(v.t1) - (int64_t)v.m1) <= cap(v.t1);
                if (ok && v.t2 < (uint32_t)tp.T) ok = (uint64_t)(mined(v.t2) + (int64_t)v.m1) <= cap(v.t2);
            }
        }
    }
    v.feasible = ok;
    return v;
}

// lo/hi bounds of block b from the current periods (1-5 pattern or CSR).
template <typename Period>
__device__ __forceinline__ uint32_t block_bounds(const Topo &tp, int32_t b, Period period) {
    uint32_t lo = 0, hi = (uint32_t)tp.T;
    if (tp.nx > 0) {
        int32_t nxy = tp.nx * tp.ny;
        int32_t x = b % tp.nx, y = (b / tp.nx) % tp.ny, z = b / nxy;
        const int dx[5] = {0, -1, 1, 0, 0};
        const int dy[5] = {0, 0, 0, -1, 1};
#pragma unroll
        for (int k = 0; k < 5; k++) {
            int32_t px = x + dx[k], py = y + dy[k];
            if (px < 0 || px >= tp.nx || py < 0 || py >= tp.ny) continue;
            if (z > 0) {
                uint32_t t = period(px + tp.nx * (py + tp.ny * (z - 1)));
                lo = t > lo ? t : lo;
            }
            if (z + 1 < tp.nz) {
                uint32_t t = period(px + tp.nx * (py + tp.ny * (z + 1)));
                hi = t < hi ? t : hi;
            }
        }
    } else {
        for (int32_t k = tp.pred_ptr[b]; k < tp.pred_ptr[b + 1]; k++) {
            uint32_t t = period(tp.pred_idx[k]);
            lo = t > lo ? t : lo;
        }
        for (int32_t k = tp.succ_ptr[b]; k < tp.succ_ptr[b + 1]; k++) {
            uint32_t t = period(tp.succ_idx[k]);
            hi = t < hi ? t : hi;
        }
    }
    return blk_pack(period(b), lo, hi);
}

}  // namespace mm
