// fused.cuh -- two pyramid levels in one kernel: the low-low band between
// them never leaves the SM.
//
// A block owns `own` columns of the level-l low-low band LL (= own/2 level
// l+1 quad columns) and a segment [R0, R1) of level l+1 quad rows.  Its
// FUSED_W1 producer warps run the level-l row pipeline (TMA-fed, as fwd_unit)
// over 60 * FUSED_W1 level-l quad columns starting 4 columns left of the block;
// they store the level-l detail bands of the rows and columns the block owns
// and write every LL row they compute, LL rows 2*R0-4 .. 2*(R1+LAG)-1, into a
// ring of FUSED_K rows in shared memory.  Its FUSED_W2 consumer warps each take
// a 128-column window of the ring, run the level l+1 row pipeline and store
// the level l+1 bands.
//
// Level l+1 needs LL extended symmetrically (whole-sample).  Columns outside
// LL are mirrored from inside the window (as load_quad_row does).  Rows
// outside LL are read from their mirror rows in the ring: LL rows that the
// producers compute past the bottom edge are half-sample mirror images when
// the level-l height is even, so they cannot be used as they are.  The
// mirror row of a row past the bottom is at most 2*(2*LAG+1) rows back, so in
// the bottom segment the consumers release ring rows that many rows late; the
// mirror rows of rows above the top are rows 1..4, read ahead of time.
//
// Each ring slot has a `full` mbarrier (one arrival per producer warp and
// row) and an `empty` one (one per consumer warp and row).  A warp waits on a
// row's `full` phase before it releases the row, so phases never alias.
// Every wait is bounded; a warp that times out sets the status word and
// returns, and the others then time out in turn.
#pragma once

#include "kernels.cuh"

namespace dwt2 {

constexpr int FUSED_K = 24;        // ring rows
constexpr int FUSED_DEFER = 10;    // late release of bottom rows: 2 * (2 * LAG + 1) for LAG <= 2
constexpr int FUSED_RING_W = 120 * (FUSED_W2 - 1) + 128;  // the last consumer window ends here
constexpr int FUSED_STAGE = 2 * FUSED_QR * 128;  // elements of one producer stage
constexpr int FUSED_THREADS = (FUSED_W1 + FUSED_W2) * 32;

constexpr size_t fused_smem_bytes() {
    return size_t(FUSED_W1) * FUSED_NST * FUSED_STAGE * 4 + size_t(FUSED_K) * FUSED_RING_W * 4 +
           size_t(FUSED_W1) * FUSED_NST * 8 + size_t(2 * FUSED_K) * 8;
}

template <class CT>
struct FusedRing {
    CT* rows;         // [FUSED_K][FUSED_RING_W], column 0 = LL column P0 - 4; producers write
                      // columns 0 .. 60 * FUSED_W1 - 1, the rest only pads the last window
    uint64_t* full;
    uint64_t* empty;
    uint32_t base;    // ring count of LL row r_lo
    int r_lo;
    __device__ __forceinline__ uint32_t idx(int y) const { return base + uint32_t(y - r_lo); }
    __device__ __forceinline__ CT* row(uint32_t g) const { return rows + (g % FUSED_K) * FUSED_RING_W; }
    // producer: wait until ring count g may be written
    __device__ __forceinline__ bool claim(uint32_t g, unsigned* status, uint64_t t) const {
        if (g < FUSED_K) return true;
        return mbar_wait_bounded(&empty[g % FUSED_K], ((g / FUSED_K) - 1) & 1u, status, t);
    }
    __device__ __forceinline__ void publish(uint32_t g, int lane) const {
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[g % FUSED_K]);
    }
    // consumer: wait until ring count g holds its row
    __device__ __forceinline__ bool acquire(uint32_t g, unsigned* status, uint64_t t) const {
        return mbar_wait_bounded(&full[g % FUSED_K], (g / FUSED_K) & 1u, status, t);
    }
    __device__ __forceinline__ void release(uint32_t g, int lane) const {
        if (lane == 0) mbar_arrive(&empty[g % FUSED_K]);
    }
};

// A producer warp: level-l quad columns [jq0, jq0 + 60), LL rows
// [r_lo, r_hi) into the ring, level-l details of rows [sr0, sr1) and quad
// columns [sc0, sc1).  Ring column 0 is LL column sc0 - 4.
template <class Pipe, class OutT>
__device__ __forceinline__ bool fused_producer(const FusedParams& P, const TmaLoader& ld, int jq0, int r_lo, int r_hi,
                                               int sr0, int sr1, int sc0, int sc1, bool active,
                                               typename Pipe::CT* bufs, uint64_t* bars, uint32_t& gstage,
                                               const FusedRing<typename Pipe::CT>& rg, int lane) {
    using CT = typename Pipe::CT;
    using R = Row<CT, 2>;
    constexpr int QL = 2, QR = FUSED_QR, NST = FUSED_NST, SPX = 128;
    const FwdParams& p = P.l1;
    if (!active) {  // no consumer reads these columns: keep the ring protocol only
        for (int y = r_lo; y < r_hi; ++y) {
            const uint32_t g = rg.idx(y);
            if (!rg.claim(g, P.status, P.timeout_ns)) return false;
            rg.publish(g, lane);
        }
        return true;
    }
    const int A0 = r_lo - 2;
    const int n_arr = (r_hi - r_lo) + 2 + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int NT = (n_arr + QR - 1) / QR;
    const int x0 = 2 * jq0 - 2 * HALO_Q;  // multiple of 4
    const int jb = x0 / 2 + QL * lane;
    const bool edge = (x0 < 0) || (x0 + SPX > p.w);
    bool mp[QL], ev[QL], dv[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        mp[q] = (lq >= HALO_Q) && (lq < 32 * QL - HALO_Q);
        const bool own = mp[q] && (jb + q >= sc0) && (jb + q < sc1);
        ev[q] = own && (jb + q < p.wq);
        dv[q] = own && (jb + q < p.wh);
    }
    const bool ring_lane = mp[0] && mp[1];  // lanes 1..30
    const int rcol = jb - (sc0 - 4);        // ring column of the lane's first quad

    int issued = 0, landed = 0;
    for (; issued < NST && issued < NT; ++issued) {
        const uint32_t gs = gstage + issued;
        ld.issue<CT, QL, QR>(bufs + (gs % NST) * FUSED_STAGE, &bars[gs % NST], x0, 2 * (A0 + issued * QR), p.h, p.w,
                             lane, P.status);
    }
    Pipe pipe;
    pipe.init();
    bool ok = true;
    const CT* stage = bufs;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            constexpr int QI = PH % QR;
            if (!ok || gi * PHASES + PH >= QR * NT) return;
            if constexpr (QI == 0) {
                const uint32_t gs = gstage + landed;
                if (!mbar_wait_bounded(&bars[gs % NST], (gs / NST) & 1u, P.status, P.timeout_ns)) {
                    ok = false;
                    return;
                }
                stage = bufs + (gs % NST) * FUSED_STAGE;
                ++landed;
            }
            const int vi = A0 + gi * PHASES + PH;
            load_quad_row<CT, QL>(stage + (2 * QI) * SPX, pipe.template slot<PH>(), lane, edge, x0, p.w);
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if (oi >= r_lo && oi < r_hi) {
                const uint32_t g = rg.idx(oi);
                if (!rg.claim(g, P.status, P.timeout_ns)) {
                    ok = false;
                    return;
                }
                if (ring_lane) st_pair<CT>(rg.row(g) + rcol, out.c1[0], out.c1[1]);
                rg.publish(g, lane);
                if (oi >= sr0 && oi < sr1) {
                    OutT* crow = reinterpret_cast<OutT*>(p.coef) + int64_t(oi) * p.coef_pitch;
                    store_pair<OutT, CT>(crow + p.wq, jb, out.c2[0], out.c2[1], dv[0], dv[1], p.vec_hi);
                    if (oi < p.hh) {
                        OutT* crow_b = reinterpret_cast<OutT*>(p.coef) + int64_t(p.hq + oi) * p.coef_pitch;
                        store_pair<OutT, CT>(crow_b, jb, out.c3[0], out.c3[1], ev[0], ev[1], p.vec_lo);
                        store_pair<OutT, CT>(crow_b + p.wq, jb, out.c4[0], out.c4[1], dv[0], dv[1], p.vec_hi);
                    }
                }
            }
            if constexpr (QI == QR - 1) {
                __syncwarp();
                if (issued < NT) {
                    const uint32_t gs = gstage + issued;
                    ld.issue<CT, QL, QR>(bufs + (gs % NST) * FUSED_STAGE, &bars[gs % NST], x0,
                                         2 * (A0 + issued * QR), p.h, p.w, lane, P.status);
                    ++issued;
                }
            }
        });
    }
    if (!ok) {
        // give the copies still in flight a bounded time to land
        for (int u = landed; u < issued; ++u) {
            const uint32_t gu = gstage + u;
            mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, P.timeout_ns);
        }
        return false;
    }
    gstage += NT;
    return true;
}

// A consumer warp: level l+1 quad rows [R0, R1) of the 60-quad strip starting
// at quad jq0 (output quads below jq_end), reading ring columns wcol ..
// wcol + 127 (LL columns 2*jq0 - 4 ..).
template <class Pipe, class OutT>
__device__ __forceinline__ bool fused_consumer(const FusedParams& P, int jq0, int jq_end, int wcol, int R0, int R1,
                                               int r_hi, const FusedRing<typename Pipe::CT>& rg, int lane) {
    using CT = typename Pipe::CT;
    using R = Row<CT, 2>;
    constexpr int QL = 2, SPX = 128;
    const FwdParams& p = P.l2;
    const bool active = jq0 < min(jq_end, p.wq);
    const int defer = (r_hi > p.h) ? FUSED_DEFER : 0;
    const int A0 = R0 - 2;
    const int n_arr = (R1 - R0) + 2 + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int x0 = 2 * jq0 - 2 * HALO_Q;
    const int jb = x0 / 2 + QL * lane;
    const bool edge = (x0 < 0) || (x0 + SPX > p.w);
    bool ev[QL], dv[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        const bool mine = (lq >= HALO_Q) && (lq < 32 * QL - HALO_Q) && (jb + q < jq_end);
        ev[q] = mine && (jb + q < p.wq);
        dv[q] = mine && (jb + q < p.wh);
    }
    Pipe pipe;
    pipe.init();
    bool ok = true;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            if (!ok || gi * PHASES + PH >= n_arr) return;
            const int vi = A0 + gi * PHASES + PH;
            const int y0 = 2 * vi, y1 = y0 + 1;
            const int s0 = fold_ws(y0, p.h), s1 = fold_ws(y1, p.h);
            if (!rg.acquire(rg.idx(y0), P.status, P.timeout_ns) || !rg.acquire(rg.idx(y1), P.status, P.timeout_ns) ||
                (s0 != y0 && !rg.acquire(rg.idx(s0), P.status, P.timeout_ns)) ||
                (s1 != y1 && !rg.acquire(rg.idx(s1), P.status, P.timeout_ns))) {
                ok = false;
                return;
            }
            R& in = pipe.template slot<PH>();
            if (active) {
                const CT* e_row = rg.row(rg.idx(s0)) + wcol;
                const CT* o_row = rg.row(rg.idx(s1)) + wcol;
                CT e[4], o[4];
                ld4_smem<CT>(e_row + 4 * lane, e);
                ld4_smem<CT>(o_row + 4 * lane, o);
                if (edge) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int px = x0 + 4 * lane + k;
                        if (px < 0 || px >= p.w) {
                            const int src = fold_ws(px, p.w) - x0;
                            const bool inw = (src >= 0) && (src < SPX);
                            e[k] = inw ? e_row[src] : CT(0);
                            o[k] = inw ? o_row[src] : CT(0);
                        }
                    }
                }
                in.c1[0] = e[0], in.c2[0] = e[1], in.c1[1] = e[2], in.c2[1] = e[3];
                in.c3[0] = o[0], in.c4[0] = o[1], in.c3[1] = o[2], in.c4[1] = o[3];
            }
            __syncwarp();
            if (y0 - defer >= rg.r_lo) rg.release(rg.idx(y0 - defer), lane);
            if (y1 - defer >= rg.r_lo) rg.release(rg.idx(y1 - defer), lane);
            if (!active) return;
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if (oi >= R0 && oi < R1) {
                if (p.ll_is_ct) {
                    CT* lrow = reinterpret_cast<CT*>(p.ll) + int64_t(oi) * p.ll_pitch;
                    store_pair<CT, CT>(lrow, jb, out.c1[0], out.c1[1], ev[0], ev[1], true);
                } else {
                    OutT* lrow = reinterpret_cast<OutT*>(p.ll) + int64_t(oi) * p.ll_pitch;
                    store_pair<OutT, CT>(lrow, jb, out.c1[0], out.c1[1], ev[0], ev[1], p.vec_ll);
                }
                OutT* crow = reinterpret_cast<OutT*>(p.coef) + int64_t(oi) * p.coef_pitch;
                store_pair<OutT, CT>(crow + p.wq, jb, out.c2[0], out.c2[1], dv[0], dv[1], p.vec_hi);
                if (oi < p.hh) {
                    OutT* crow_b = reinterpret_cast<OutT*>(p.coef) + int64_t(p.hq + oi) * p.coef_pitch;
                    store_pair<OutT, CT>(crow_b, jb, out.c3[0], out.c3[1], ev[0], ev[1], p.vec_lo);
                    store_pair<OutT, CT>(crow_b + p.wq, jb, out.c4[0], out.c4[1], dv[0], dv[1], p.vec_hi);
                }
            }
        });
    }
    if (!ok) return false;
    for (int y = max(rg.r_lo, r_hi - defer); y < r_hi; ++y) rg.release(rg.idx(y), lane);
    return true;
}

template <class Pipe, class OutT>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
    fused2_kernel(const __grid_constant__ CUtensorMap tm_box, const __grid_constant__ CUtensorMap tm_row,
                  const FusedParams P) {
    using CT = typename Pipe::CT;
    constexpr int W1 = FUSED_W1, NST = FUSED_NST;
    extern __shared__ __align__(128) unsigned char smem[];
    CT* stages = reinterpret_cast<CT*>(smem);
    CT* ring_rows = stages + size_t(W1) * NST * FUSED_STAGE;
    uint64_t* tma_bars = reinterpret_cast<uint64_t*>(ring_rows + size_t(FUSED_K) * FUSED_RING_W);
    uint64_t* full = tma_bars + W1 * NST;
    uint64_t* empty = full + FUSED_K;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < W1 * NST; ++i) mbar_init(&tma_bars[i], TmaLoader::ARRIVALS);
        for (int i = 0; i < FUSED_K; ++i) {
            mbar_init(&full[i], FUSED_W1);
            mbar_init(&empty[i], FUSED_W2);
        }
        fence_mbar_init();
        tma_prefetch_desc(&tm_box);
        tma_prefetch_desc(&tm_row);
    }
    __syncthreads();

    const TmaLoader ld{&tm_box, &tm_row};
    CT* bufs = stages + size_t(warp < W1 ? warp : 0) * NST * FUSED_STAGE;
    uint64_t* bars = tma_bars + (warp < W1 ? warp : 0) * NST;
    uint32_t gstage = 0, gring = 0;
    const int hq2 = P.l2.hq, wq1 = P.l2.w;
    for (int item = blockIdx.x; item < P.n_items; item += gridDim.x) {
        const int c = item % P.n_cols, g2 = item / P.n_cols;
        const int R0 = g2 * P.seg2;
        const int R1 = (g2 == P.n_segs - 1) ? hq2 : R0 + P.seg2;
        const int r_lo = 2 * R0 - 4, r_hi = 2 * (R1 + Pipe::LAG);
        const int P0 = P.own * c;
        const FusedRing<CT> rg{ring_rows, full, empty, gring, r_lo};
        bool ok;
        if (warp < W1) {
            const int jq0 = P0 - 4 + 60 * warp;
            const bool active = jq0 < min(P0 + P.own + 4, wq1);
            ok = fused_producer<Pipe, OutT>(P, ld, jq0, r_lo, r_hi, 2 * R0, min(2 * R1, P.l1.hq), P0, P0 + P.own,
                                            active, bufs, bars, gstage, rg, lane);
        } else {
            const int j = warp - W1;
            const int jq0 = P0 / 2 + 60 * j;
            ok = fused_consumer<Pipe, OutT>(P, jq0, (P0 + P.own) / 2, 120 * j, R0, R1, r_hi, rg, lane);
        }
        if (!ok) return;
        gring += uint32_t(r_hi - r_lo);
    }
}

}  // namespace dwt2
