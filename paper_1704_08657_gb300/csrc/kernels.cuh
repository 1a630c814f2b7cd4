// kernels.cuh -- the transform kernels of one pyramid level.
//
// Work decomposition: the level is cut into vertical strips of 32*QL - 4
// output quads (a warp loads 64*QL pixels; 4 on each side are halo) and
// horizontal segments of seg_rows output quad rows.  One (strip, segment)
// pair is a unit of work for one warp.  A warp streams the quad rows of its
// unit top to bottom through the row pipeline of the scheme (schemes.cuh),
// starting two quad rows above the segment (warm-up) and running LAG rows
// past it, in groups of PHASES arrivals unrolled at compile time.
//
// Forward: each warp owns a ring of NST shared-memory stages of QR quad rows
// (2*QR pixel rows x 64*QL pixels) filled by 2-D TMA loads that complete on
// one mbarrier per stage; lane 0 refills a stage once the warp has read it.
// Rows outside the image are fetched from their whole-sample mirror rows (one
// single-row TMA box per pixel row); columns outside the image are mirrored in
// shared memory by the edge strips.  With the symmetric extension in place the
// lifting needs no boundary cases: every step preserves the symmetry, so the
// exact per-step mirrored result appears inside the image.
//
// Inverse and adjoint: the four bands are read into a ring of shared-memory
// stages, two quad rows ahead of the pipeline.  The inverse reads mirrored band
// positions at the edges (the extension of the coefficients that the symmetric
// image extension produces); the adjoint reads zeros there, runs on the
// extended domain two quads past every edge and folds the extended outputs
// back onto their mirrors (Adj97, adj_fold_kernel).
#pragma once

#include <type_traits>
#include <utility>

#include "schemes.cuh"

namespace dwt2 {

// compile-time loop: f(std::integral_constant<int, 0>) ... f(<N-1>)
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <class CT>
__device__ __forceinline__ void ld4_smem(const CT* p, CT* v) {
    if constexpr (std::is_same<CT, float>::value) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
        const int4 t = *reinterpret_cast<const int4*>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
}

template <class CT>
__device__ __forceinline__ void st4(CT* p, CT a, CT b, CT c, CT d) {
    if constexpr (std::is_same<CT, float>::value)
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    else
        *reinterpret_cast<int4*>(p) = make_int4(a, b, c, d);
}

// The pieces of work of one warp, as (strip, first quad row, end quad row):
// balanced mode gives each warp one contiguous range of the strip-major quad
// rows (split where it crosses a strip end); otherwise fixed units of
// seg_rows rows are dealt round-robin.
template <class P>
struct Pieces {
    int64_t rb, re;
    int unit, stride;
    __device__ __forceinline__ Pieces(const P& p, int wg, int nwarps) {
        const int64_t T = int64_t(p.n_strips) * p.hq;
        rb = T * wg / nwarps;
        re = T * (wg + 1) / nwarps;
        unit = wg;
        stride = nwarps;
    }
    __device__ __forceinline__ bool next(const P& p, int& s, int& R0, int& R1) {
        if (p.balanced) {
            if (rb >= re) return false;
            s = int(rb / p.hq);
            R0 = int(rb - int64_t(s) * p.hq);
            R1 = int(min(int64_t(p.hq), R0 + (re - rb)));
            rb += R1 - R0;
            return true;
        }
        if (unit >= p.n_units) return false;
        s = unit % p.n_strips;
        R0 = (unit / p.n_strips) * p.seg_rows;
        R1 = min(R0 + p.seg_rows, p.hq);
        unit += stride;
        return true;
    }
};

// shared-memory bytes of a forward launch
template <int QL, int QR, int NST, int NW>
constexpr size_t fwd_smem_bytes() {
    return size_t(NW) * NST * (2 * QR * 64 * QL * 4) + size_t(NW) * NST * 8;
}

// One quad row (two pixel rows) of the lane from a shared-memory stage; edge
// strips replace pixels outside [0, w) by their mirror images.
template <class CT, int QL>
__device__ __forceinline__ void load_quad_row(const CT* s0, Row<CT, QL>& r, int lane, bool edge, int x0, int w) {
    constexpr int SPX = 64 * QL;
    const CT* s1 = s0 + SPX;
    CT e[2 * QL], o[2 * QL];
#pragma unroll
    for (int k = 0; k < 2 * QL; k += 4) {
        ld4_smem<CT>(s0 + 2 * QL * lane + k, e + k);
        ld4_smem<CT>(s1 + 2 * QL * lane + k, o + k);
    }
    if (edge) {
#pragma unroll
        for (int k = 0; k < 2 * QL; ++k) {
            const int px = x0 + 2 * QL * lane + k;
            if (px < 0 || px >= w) {
                const int src = fold_ws(px, w) - x0;
                const bool in = (src >= 0) && (src < SPX);
                e[k] = in ? s0[src] : CT(0);
                o[k] = in ? s1[src] : CT(0);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        r.c1[q] = e[2 * q];
        r.c2[q] = e[2 * q + 1];
        r.c3[q] = o[2 * q];
        r.c4[q] = o[2 * q + 1];
    }
}

// Edge strips of the forward: once a stage has landed, every pixel of the
// lane outside [0, w) takes the value of its whole-sample mirror in place
// (zero where the mirror lies outside the strip, beyond the filter support of
// any stored output).  Sources are pixels inside the image, which no lane
// rewrites, so the lanes need no barrier between them; the proxy fence orders
// these generic writes before the next asynchronous fill of the stage.  Not
// inlined: the row loop of interior strips stays as small as it was.
template <class CT, int QL>
__device__ __noinline__ void fwd_fix_edges(CT* stage, int rows, int x0, int w, int lane) {
    constexpr int SPX = 64 * QL;
    for (int k = 0; k < 2 * QL; ++k) {
        const int px = x0 + 2 * QL * lane + k;
        if (px >= 0 && px < w) continue;
        const int src = fold_ws(px, w) - x0;
        const bool in = (src >= 0) && (src < SPX);
        for (int r = 0; r < rows; ++r) {
            CT* row = stage + r * SPX;
            row[2 * QL * lane + k] = in ? row[src] : CT(0);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ loaders
// A loader fills one shared-memory stage (2*QR pixel rows of 64*QL pixels,
// starting at pixel column x0 and pixel row y0 of the level's input) and
// makes it complete on the stage's mbarrier.  Rows outside [0, h) are taken
// from their whole-sample mirror rows; columns outside [0, w) are left as
// zeros (load_quad_row mirrors them).

// 2-D TMA (cp.async.bulk.tensor) issued by lane 0; one box when every row is
// inside the image, else one single-row box per pixel row.
struct TmaLoader {
    static constexpr unsigned ARRIVALS = 1;
    const CUtensorMap* box;
    const CUtensorMap* row;
    template <class CT, int QL, int QR>
    __device__ __forceinline__ void issue(CT* dst, uint64_t* bar, int x0, int y0, int h, int /*w*/, int lane,
                                          unsigned* status) const {
        constexpr int SPX = 64 * QL, ROWS = 2 * QR;
        if (lane != 0) return;
        // the box's first column on a 16-byte boundary (columns outside the
        // image are TMA's zero fill, checked by the hardware)
        if (!dev_in(status, (x0 & 3) == 0)) x0 &= ~3;
        mbar_expect_tx(bar, unsigned(ROWS * SPX * 4));
        if (y0 >= 0 && y0 + ROWS <= h) {
            tma_load_2d(dst, box, x0, y0, bar);
        } else {
#pragma unroll 1
            for (int r = 0; r < ROWS; ++r) {
                int y = fold_ws(y0 + r, h);
                if (!dev_in(status, y >= 0 && y < h)) y = 0;
                tma_load_2d(dst + r * SPX, row, x0, y, bar);
            }
        }
    }
};

// 16-byte cp.async by every lane (one 4-pixel chunk per lane per row and QL/2
// chunks per lane), zero-filling the part of a chunk past the right edge; each
// lane's copies arrive on the mbarrier when they land.  Needs a 16-byte
// aligned source row (pitch a multiple of 4 elements).
template <class CT>
struct CpAsyncLoader {
    static constexpr unsigned ARRIVALS = 32;
    const CT* src;
    int64_t pitch;
    template <class CT_, int QL, int QR>
    __device__ __forceinline__ void issue(CT_* dst, uint64_t* bar, int x0, int y0, int h, int w, int lane,
                                          unsigned* status) const {
        constexpr int SPX = 64 * QL, ROWS = 2 * QR;
        const bool inside = (y0 >= 0) && (y0 + ROWS <= h);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            int y = inside ? y0 + r : fold_ws(y0 + r, h);
            if (!dev_in(status, y >= 0 && y < h)) y = 0;
            const CT* srow = src + int64_t(y) * pitch;
#pragma unroll
            for (int k = 0; k < QL / 2; ++k) {
                const int c = lane + 32 * k;  // chunk index in the strip
                const int px = x0 + 4 * c;
                int n = (px >= 0) ? max(0, min(4, w - px)) : 0;
                if (!dev_in(status, n == 0 || (px >= 0 && px + n <= w))) n = 0;
                const CT* g = srow + (n > 0 ? px : 0);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + r * SPX + 4 * c)),
                             "l"(g), "r"(4 * n)
                             : "memory");
            }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
};

// ------------------------------------------------------------------ forward
// One unit of work: quad rows [R0, R1) of strip s of one level.  P provides
// the level's geometry and outputs (fields of FwdParams); bufs / bars are the
// warp's stage ring, gstage the warp's running stage count (slot and mbarrier
// phase).  Returns false when a stage wait timed out.
//
// MODE 0 handles every strip.  MODE 1 and 2 are compiled for strips whose
// band rows all take paired stores (fwd_pairs_ok), with the low-low band in
// the compute type (1) or the coefficient type (2): their row loop has no
// store-alignment branches, which keeps the hot loop small in the instruction
// cache.  Edge strips run the same row loop as interior ones: their mirrored
// columns are filled in the stage (fwd_fix_edges) and per-lane masks drop the
// quads outside the bands.
template <class P>
__device__ __forceinline__ bool fwd_pairs_ok(const P& p, int x0, int QL, int halo) {
    // every pair starts at an even quad: with both band widths even no pair
    // straddles a band's last column; otherwise the strip must end inside both
    return p.vec_lo && p.vec_hi && (p.ll_is_ct || p.vec_ll) &&
           ((p.wq % 2 == 0 && p.wh % 2 == 0) || (x0 / 2 + 32 * QL - halo <= p.wh));
}

template <class Pipe, class OutT, int QL, int QR, int NST, int MODE = 0, class P, class Loader>
__device__ __forceinline__ bool fwd_unit(const P& p, const Loader& ld, int s, int R0, int R1,
                                         typename Pipe::CT* bufs, uint64_t* bars, uint32_t& gstage, int lane) {
    using CT = typename Pipe::CT;
    using R = Row<CT, QL>;
    constexpr int SPX = 64 * QL;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int OUTQ = 32 * QL - 2 * HQ;
    constexpr int ROWS = 2 * QR;
    constexpr int STAGE_ELEMS = ROWS * SPX;
    static_assert(PHASES % QR == 0, "a group of arrivals must cover whole stages");
    static_assert(QL % 2 == 0, "band stores go in pairs");

    const int A0 = R0 - WARM;                         // first quad row streamed
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;   // quad rows streamed
    const int n_grp = (n_arr + PHASES - 1) / PHASES;  // groups of arrivals (the last may stop early)
    const int NT = (n_arr + QR - 1) / QR;             // stages
    const int x0 = s * (2 * OUTQ) - 2 * HQ;           // first pixel (multiple of 4)
    const int jb = x0 / 2 + QL * lane;                // first quad column of the lane
    constexpr bool SPEC = MODE != 0;
    const bool edge = (x0 < 0) || (x0 + SPX > p.w);
    const bool llct = MODE == 1 ? true : (MODE == 2 ? false : bool(p.ll_is_ct));

    // which of the lane's quads this strip outputs, per band parity
    bool ev[QL], dv[QL], mp[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        mp[q] = (lq >= HQ) && (lq < 32 * QL - HQ);
        ev[q] = mp[q] && (jb + q < p.wq);
        dv[q] = mp[q] && (jb + q < p.wh);
    }
    // paired stores: both quads of the pair output by this strip and inside
    // the even-column (LL, LH) or odd-column (HL, HH) bands
    bool pe[QL / 2], po[QL / 2];
#pragma unroll
    for (int q = 0; q < QL; q += 2) {
        pe[q / 2] = mp[q] && mp[q + 1] && (jb + q + 1 < p.wq);
        po[q / 2] = mp[q] && mp[q + 1] && (jb + q + 1 < p.wh);
    }
    // warp-uniform: every band row takes paired stores
    const bool fast = SPEC ? true : fwd_pairs_ok(p, x0, QL, HQ);
    // band pointers at output row R0, advanced one pitch per stored row
    OutT* hl = reinterpret_cast<OutT*>(p.coef) + int64_t(R0) * p.coef_pitch + p.wq + jb;
    OutT* lh = reinterpret_cast<OutT*>(p.coef) + int64_t(p.hq + R0) * p.coef_pitch + jb;
    OutT* hh = lh + p.wq;
    CT* llc = reinterpret_cast<CT*>(p.ll) + int64_t(R0) * p.ll_pitch + jb;
    OutT* llo = reinterpret_cast<OutT*>(p.ll) + int64_t(R0) * p.ll_pitch + jb;
    // checked build: the four bands as rectangles (LL hq x wq, HL hq x wh,
    // LH hh x wq, HH hh x wh) that every store must fall in
    const OutT* hl0 = reinterpret_cast<const OutT*>(p.coef) + p.wq;
    const OutT* lh0 = reinterpret_cast<const OutT*>(p.coef) + int64_t(p.hq) * p.coef_pitch;
    const OutT* hh0 = lh0 + p.wq;
    const CT* llc0 = reinterpret_cast<const CT*>(p.ll);
    const OutT* llo0 = reinterpret_cast<const OutT*>(p.ll);
    auto in_band = [&](const auto* ptr, const auto* base, int64_t pitch, int rows, int cols, bool m0, bool m1) {
        return (!m0 || dev_in_rect(p.status, ptr, base, pitch, rows, cols, 1)) &&
               (!m1 || dev_in_rect(p.status, ptr + 1, base, pitch, rows, cols, 1));
    };

    for (int t = 0; t < NST && t < NT; ++t) {
        const uint32_t gs = gstage + t;
        ld.template issue<CT, QL, QR>(bufs + (gs % NST) * STAGE_ELEMS, &bars[gs % NST], x0, 2 * (A0 + t * QR), p.h,
                                      p.w, lane, p.status);
    }

    Pipe pipe;
    pipe.init();
    bool ok = true;
    int t = 0, slot = 0;
    const CT* stage = bufs;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            constexpr int QI = PH % QR;
            if (gi * PHASES + PH >= QR * NT) return;  // past the unit's last stage
            if constexpr (QI == 0) {
                if (!ok) return;
                const uint32_t gs = gstage + t;
                slot = gs % NST;
                if (!mbar_wait_bounded(&bars[slot], (gs / NST) & 1u, p.status, p.timeout_ns)) {
                    // give the copies still in flight a bounded time to land
                    for (int u = t + 1; u < NT && u < t + NST; ++u) {
                        const uint32_t gu = gstage + u;
                        mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, p.timeout_ns);
                    }
                    ok = false;
                    return;
                }
                stage = bufs + slot * STAGE_ELEMS;
                if (edge) fwd_fix_edges<CT, QL>(const_cast<CT*>(stage), ROWS, x0, p.w, lane);
            }
            const int vi = A0 + gi * PHASES + PH;  // quad row streamed now
            load_quad_row<CT, QL>(stage + (2 * QI) * SPX, pipe.template slot<PH>(), lane, false, x0, p.w);
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            const bool row_on = (oi >= R0) & (oi < R1);
            const bool orow = row_on & (oi < p.hh);
            if (fast) {
#pragma unroll
                for (int q = 0; q < QL; q += 2) {
                    bool on_e = row_on & pe[q / 2], on_o = row_on & po[q / 2];
                    bool oo_e = orow & pe[q / 2], oo_o = orow & po[q / 2];
                    if constexpr (CHECKED_BUILD) {
                        on_e = on_e && (llct ? in_band(llc + q, llc0, p.ll_pitch, p.hq, p.wq, true, true)
                                             : in_band(llo + q, llo0, p.ll_pitch, p.hq, p.wq, true, true));
                        on_o = on_o && in_band(hl + q, hl0, p.coef_pitch, p.hq, p.wh, true, true);
                        oo_e = oo_e && in_band(lh + q, lh0, p.coef_pitch, p.hh, p.wq, true, true);
                        oo_o = oo_o && in_band(hh + q, hh0, p.coef_pitch, p.hh, p.wh, true, true);
                    }
                    if (llct) {
                        if (on_e) st_pair<CT>(llc + q, out.c1[q], out.c1[q + 1]);
                    } else {
                        if (on_e) st_pair<OutT>(llo + q, Cvt<OutT>::to(out.c1[q]), Cvt<OutT>::to(out.c1[q + 1]));
                    }
                    if (on_o) st_pair<OutT>(hl + q, Cvt<OutT>::to(out.c2[q]), Cvt<OutT>::to(out.c2[q + 1]));
                    if (oo_e) st_pair<OutT>(lh + q, Cvt<OutT>::to(out.c3[q]), Cvt<OutT>::to(out.c3[q + 1]));
                    if (oo_o) st_pair<OutT>(hh + q, Cvt<OutT>::to(out.c4[q]), Cvt<OutT>::to(out.c4[q + 1]));
                }
            } else if (row_on) {
#pragma unroll
                for (int q = 0; q < QL; q += 2) {
                    bool ok_l = true, ok_hl = true, ok_lh = true, ok_hh = true;
                    if constexpr (CHECKED_BUILD) {
                        ok_l = llct ? in_band(llc + q, llc0, p.ll_pitch, p.hq, p.wq, ev[q], ev[q + 1])
                                    : in_band(llo + q, llo0, p.ll_pitch, p.hq, p.wq, ev[q], ev[q + 1]);
                        ok_hl = in_band(hl + q, hl0, p.coef_pitch, p.hq, p.wh, dv[q], dv[q + 1]);
                        ok_lh = !orow || in_band(lh + q, lh0, p.coef_pitch, p.hh, p.wq, ev[q], ev[q + 1]);
                        ok_hh = !orow || in_band(hh + q, hh0, p.coef_pitch, p.hh, p.wh, dv[q], dv[q + 1]);
                    }
                    if (llct) {
                        if (ok_l) store_pair<CT, CT>(llc, q, out.c1[q], out.c1[q + 1], ev[q], ev[q + 1], true);
                    } else if (ok_l) {
                        store_pair<OutT, CT>(llo, q, out.c1[q], out.c1[q + 1], ev[q], ev[q + 1], p.vec_ll);
                    }
                    if (ok_hl) store_pair<OutT, CT>(hl, q, out.c2[q], out.c2[q + 1], dv[q], dv[q + 1], p.vec_hi);
                    if (orow) {
                        if (ok_lh) store_pair<OutT, CT>(lh, q, out.c3[q], out.c3[q + 1], ev[q], ev[q + 1], p.vec_lo);
                        if (ok_hh) store_pair<OutT, CT>(hh, q, out.c4[q], out.c4[q + 1], dv[q], dv[q + 1], p.vec_hi);
                    }
                }
            }
            const int64_t cstep = row_on ? p.coef_pitch : 0;
            const int64_t lstep = row_on ? p.ll_pitch : 0;
            hl += cstep;
            lh += cstep;
            hh += cstep;
            llc += lstep;
            llo += lstep;
            if constexpr (QI == QR - 1) {
                __syncwarp();
                if (ok && t + NST < NT)
                    ld.template issue<CT, QL, QR>(bufs + slot * STAGE_ELEMS, &bars[slot], x0,
                                                  2 * (A0 + (t + NST) * QR), p.h, p.w, lane, p.status);
                ++t;
            }
        });
    }
    if (ok) gstage += NT;
    return ok;
}

template <class CT, int QL, int QR, int NST, int NW>
__device__ __forceinline__ void stage_ring(unsigned char* smem, int warp, CT*& bufs, uint64_t*& bars) {
    constexpr int STAGE_ELEMS = 2 * QR * 64 * QL;
    bufs = reinterpret_cast<CT*>(smem) + warp * NST * STAGE_ELEMS;
    bars = reinterpret_cast<uint64_t*>(smem + size_t(NW) * NST * STAGE_ELEMS * 4) + warp * NST;
}

// Inter-level overlap.  A unit of quad rows [R0, R1) streams input rows
// 2*R0-4 .. 2*(R1+LAG+QR-2)+1 (warm-up, pipeline lag, stage rounding), folded
// into [0, h) by the symmetric extension; lane 0 waits (bounded) until every
// previous-level segment holding such a row has all its strips complete, then
// orders its later TMA reads after what it observed.
template <int LAG, int QR, int WARM>
__device__ __forceinline__ bool fwd_wait_inputs(const FwdParams& p, int R0, int R1, int lane) {
    bool ok = true;
    if (lane == 0) {
        int lo = max(0, 2 * (R0 - WARM));
        const int end = 2 * (R1 + LAG + QR - 2) + 2;  // one past the last streamed row
        const int hi = min(p.h, end);
        if (end > p.h) lo = max(0, min(lo, 2 * p.h - 1 - end));  // mirrored rows past the bottom
        for (int g = lo / p.dep_seg; g <= (hi - 1) / p.dep_seg && ok; ++g) {
            const unsigned* c = p.dep_ctr + g;
            if (ld_acquire(c) >= unsigned(p.dep_need)) continue;
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire(c) < unsigned(p.dep_need)) {
                if (globaltimer_ns() - t0 > p.timeout_ns) {
                    ok = false;
                    break;
                }
                __nanosleep(128);
            }
        }
        if (!ok && p.status) atomicOr(p.status, DEV_TIMEOUT);
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    return __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
}

// after a unit's stores: count the unit in its segment with a release
// reduction (the warp barrier orders every lane's stores before lane 0's
// release); the consumer acquires the count and fences its async proxy
__device__ __forceinline__ void fwd_signal(unsigned* ctr, int lane) {
    __syncwarp();
    if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// One pyramid level, TMA-fed: the warps take their units from Pieces.  SPEC
// compiles the specialised row loops for interior strips as well.
// Register budget of the forward kernels: the lifting pipelines in 4-warp
// blocks are held to five resident blocks per SM (at most 102 registers; the
// 5-level 16384^2 pyramid measured ~1 % faster than with four), the other
// pipelines and block sizes are left to the compiler.
template <class Pipe, int NW>
struct FwdMinBlocks {
    static constexpr int value = 1;
};
template <int S, int QL>
struct FwdMinBlocks<Fwd97<S, QL>, 4> {
    static constexpr int value = 5;
};
template <int S, int QL>
struct FwdMinBlocks<Fwd53<S, QL>, 4> {
    static constexpr int value = 5;
};

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value)
    fwd_tma_kernel(const __grid_constant__ CUtensorMap tm_box, const __grid_constant__ CUtensorMap tm_row,
                   const FwdParams p) {
    using CT = typename Pipe::CT;
    constexpr int HQ = PipeGeom<Pipe>::HALO;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TmaLoader::ARRIVALS);
        fence_mbar_init();
        tma_prefetch_desc(&tm_box);
        tma_prefetch_desc(&tm_row);
    }
    __syncwarp();
    // the input (the previous level's low-low band) and the outputs are only
    // touched after the previous grid in the stream has completed, or, with
    // inter-level overlap, after the segments a unit reads are complete
    if (p.dep_ctr == nullptr) griddep_wait();
    griddep_launch_dependents();
    const TmaLoader ld{&tm_box, &tm_row};
    uint32_t gstage = 0;
    Pieces<FwdParams> pieces(p, blockIdx.x * NW + warp, gridDim.x * NW);
    int s, R0, R1;
    while (pieces.next(p, s, R0, R1)) {
        if (p.dep_ctr != nullptr && !fwd_wait_inputs<Pipe::LAG, QR, PipeGeom<Pipe>::WARM>(p, R0, R1, lane)) return;
        bool ok;
        if constexpr (SPEC) {
            if (fwd_pairs_ok(p, s * (2 * (32 * QL - 2 * HQ)) - 2 * HQ, QL, HQ))
                ok = p.ll_is_ct ? fwd_unit<Pipe, OutT, QL, QR, NST, 1>(p, ld, s, R0, R1, bufs, bars, gstage, lane)
                                : fwd_unit<Pipe, OutT, QL, QR, NST, 2>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
            else
                ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        } else {
            ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok || dev_check_tripped(p.status)) return;
        if (p.out_ctr != nullptr && !(p.test_drop && s == 0 && R0 == 0)) fwd_signal(p.out_ctr + R0 / p.seg_rows, lane);
    }
}

// One level of a group of images (GroupLaunch): the warps take units in order,
// find their image by a binary search over the group's unit ranges, and run
// the single-image row loop with that image's parameters and tensor maps.
// Launches of one level touch disjoint images, so only the first launch of a
// level waits for what came before it; the others start as soon as the
// previous launch has placed all its blocks.
template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value)
    fwd_group_kernel(const __grid_constant__ GroupLaunch L) {
    using CT = typename Pipe::CT;
    constexpr int HQ = PipeGeom<Pipe>::HALO;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TmaLoader::ARRIVALS);
        fence_mbar_init();
    }
    __syncwarp();
    if (L.wait_prev) griddep_wait();
    griddep_launch_dependents();
    uint32_t gstage = 0;
    const int stride = gridDim.x * NW;
    for (int u = blockIdx.x * NW + warp; u < L.n_units; u += stride) {
        int lo = 0, hi = L.n_img - 1;  // the last image whose u_begin <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.img[mid].u_begin <= u) lo = mid;
            else hi = mid - 1;
        }
        const FwdParams& p = L.img[lo].p;
        const int lu = u - L.img[lo].u_begin;
        const int s = lu % p.n_strips;
        const int R0 = (lu / p.n_strips) * p.seg_rows;
        const int R1 = min(R0 + p.seg_rows, p.hq);
        const TmaLoader ld{&L.maps[2 * lo], &L.maps[2 * lo + 1]};
        if (lane == 0) {
            tma_prefetch_desc(ld.box);
            tma_prefetch_desc(ld.row);
        }
        bool ok;
        if constexpr (SPEC) {
            if (fwd_pairs_ok(p, s * (2 * (32 * QL - 2 * HQ)) - 2 * HQ, QL, HQ))
                ok = p.ll_is_ct ? fwd_unit<Pipe, OutT, QL, QR, NST, 1>(p, ld, s, R0, R1, bufs, bars, gstage, lane)
                                : fwd_unit<Pipe, OutT, QL, QR, NST, 2>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
            else
                ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        } else {
            ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok || dev_check_tripped(p.status)) return;
    }
}

// ------------------------------------------------- persistent (batched) forward
// All units of all images and levels of a plan in one launch.  Units are taken
// from a device queue in the plan's order; a unit of level l first waits
// (bounded) until the level l-1 segments it reads are complete, i.e. their
// counters reached the strip count; after its stores it bumps the counter of
// its own segment.  The queue order puts every unit about one GPU round behind
// the segments it depends on, so waits are rare and the low-low band it reads
// was written moments before (usually still in L2).

// the geometry and outputs of one unit's level, with the field names fwd_unit uses
struct PmlView {
    int h, w, hq, wq, hh, wh;
    void* coef;
    int64_t coef_pitch;
    void* ll;
    int64_t ll_pitch;
    int ll_is_ct;
    int vec_lo, vec_hi, vec_ll;
    unsigned* status;
    uint64_t timeout_ns;
};

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool TMA>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value) pml_kernel(const __grid_constant__ PmlLaunch L) {
    using CT = typename Pipe::CT;
    const PmlParams& P = L.base;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TMA ? TmaLoader::ARRIVALS : CpAsyncLoader<CT>::ARRIVALS);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t gstage = 0;
    for (;;) {
        int u = 0;
        if (lane == 0) u = int(atomicAdd(P.queue, 1u));
        u = __shfl_sync(FULL, u, 0);
        if (u >= P.n_units) break;
        const PmlUnit un = P.units[u];
        const PmlDesc& d = P.descs[un.desc];
        if (d.dep_base >= 0) {
            bool waited_ok = true;
            if (lane == 0) {
                for (int g = un.dep_lo; g <= un.dep_hi; ++g) {
                    const unsigned* c = P.counters + d.dep_base + g;
                    if (ld_acquire(c) >= unsigned(d.dep_need)) continue;
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_acquire(c) < unsigned(d.dep_need)) {
                        if (globaltimer_ns() - t0 > P.timeout_ns) {
                            waited_ok = false;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                if (!waited_ok && P.status) atomicOr(P.status, DEV_TIMEOUT);
                // the level's input was written through the generic proxy by other
                // warps; TMA reads through the async proxy
                if (TMA) asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncwarp();
        }
        PmlView v;
        v.h = d.h, v.w = d.w, v.hq = d.hq, v.wq = d.wq, v.hh = d.hh, v.wh = d.wh;
        v.coef = static_cast<OutT*>(P.coef) + d.coef_off;
        v.coef_pitch = d.coef_pitch;
        v.ll = d.ll_is_ct ? static_cast<void*>(static_cast<CT*>(P.ws) + d.ll_off)
                          : static_cast<void*>(static_cast<OutT*>(P.coef) + d.ll_off);
        v.ll_pitch = d.ll_pitch;
        v.ll_is_ct = d.ll_is_ct;
        v.vec_lo = d.vec_lo && P.coef_vec, v.vec_hi = d.vec_hi && P.coef_vec;
        v.vec_ll = d.ll_is_ct ? 1 : (d.vec_ll && P.coef_vec);
        v.status = P.status;
        v.timeout_ns = P.timeout_ns;
        const int R0 = un.g * d.seg_rows;
        const int R1 = min(R0 + d.seg_rows, d.hq);
        bool ok;
        if constexpr (TMA) {
            const TmaLoader ld{L.maps + 2 * un.desc, L.maps + 2 * un.desc + 1};
            if (lane == 0) {
                tma_prefetch_desc(ld.box);
                tma_prefetch_desc(ld.row);
            }
            ok = fwd_unit<Pipe, OutT, QL, QR, NST>(v, ld, un.s, R0, R1, bufs, bars, gstage, lane);
        } else {
            const CT* src = d.src_is_ws ? static_cast<const CT*>(P.ws) + d.src_off
                                        : static_cast<const CT*>(P.in) + d.src_off;
            const CpAsyncLoader<CT> ld{src, d.src_pitch};
            ok = fwd_unit<Pipe, OutT, QL, QR, NST>(v, ld, un.s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok || dev_check_tripped(P.status)) return;
        // this unit's stores must be visible to the TMA reads of later units
        if (TMA) asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncwarp();
        if (lane == 0 && !(P.test_drop_signal && u == 0)) {
            __threadfence();
            atomicAdd(P.counters + d.ctr_base + un.g, 1u);
        }
    }
}

// ------------------------------------------------- band loads (inverse, adjoint)
template <class T>
__device__ __forceinline__ void ld_pair(const T* p, float& a, float& b, bool vec) {
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float2 t = *reinterpret_cast<const float2*>(p);
            a = t.x, b = t.y;
        } else if constexpr (std::is_same<T, __half>::value) {
            const __half2 t = *reinterpret_cast<const __half2*>(p);
            a = __low2float(t), b = __high2float(t);
        } else {
            const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(p);
            a = __low2float(t), b = __high2float(t);
        }
    } else {
        a = Cvt<T>::from(p[0]);
        b = Cvt<T>::from(p[1]);
    }
}
__device__ __forceinline__ void ld_pair(const int* p, int& a, int& b, bool vec) {
    if (vec) {
        const int2 t = *reinterpret_cast<const int2*>(p);
        a = t.x, b = t.y;
    } else {
        a = p[0];
        b = p[1];
    }
}

template <class T, class CT>
__device__ __forceinline__ CT ld_one(const T* p) {
    return CT(Cvt<T>::from(*p));
}

// One quad row of the lane's quads from the four bands.  MIRROR: positions
// outside the image read their mirror images; otherwise they read zero.
template <class CT, class BT, bool MIRROR, int QL>
__device__ __forceinline__ void load_bands(const InvParams& p, int vi, int jb, bool fast, Row<CT, QL>& r) {
    const BT* coef = reinterpret_cast<const BT*>(p.coef);
    if (fast) {  // whole strip and row inside the bands: direct pair loads
        const int64_t re = vi, ro = vi;
        const BT* hl = coef + re * p.coef_pitch + p.wq + jb;
        const BT* lh = coef + (p.hq + ro) * p.coef_pitch + jb;
        const BT* hh = lh + p.wq;
        if constexpr (CHECKED_BUILD) {
            const bool ok =
                (p.ll_is_ct ? dev_in_rect(p.status, reinterpret_cast<const CT*>(p.ll) + re * p.ll_pitch + jb,
                                          reinterpret_cast<const CT*>(p.ll), p.ll_pitch, p.hq, p.wq, QL)
                            : dev_in_rect(p.status, reinterpret_cast<const BT*>(p.ll) + re * p.ll_pitch + jb,
                                          reinterpret_cast<const BT*>(p.ll), p.ll_pitch, p.hq, p.wq, QL)) &&
                dev_in_rect(p.status, hl, coef + p.wq, p.coef_pitch, p.hq, p.wh, QL) &&
                dev_in_rect(p.status, lh, coef + int64_t(p.hq) * p.coef_pitch, p.coef_pitch, p.hh, p.wq, QL) &&
                dev_in_rect(p.status, hh, coef + int64_t(p.hq) * p.coef_pitch + p.wq, p.coef_pitch, p.hh, p.wh, QL);
            if (!ok) return;  // the row keeps its previous values; the status word has DEV_CHECK
        }
#pragma unroll
        for (int q = 0; q < QL; q += 2) {
            if (p.ll_is_ct) {
                const CT* ll = reinterpret_cast<const CT*>(p.ll) + re * p.ll_pitch + jb;
                ld_pair(ll + q, r.c1[q], r.c1[q + 1], p.vec_ll);
            } else {
                const BT* ll = reinterpret_cast<const BT*>(p.ll) + re * p.ll_pitch + jb;
                ld_pair(ll + q, r.c1[q], r.c1[q + 1], p.vec_ll);
            }
            ld_pair(hl + q, r.c2[q], r.c2[q + 1], p.vec_in_hi);
            ld_pair(lh + q, r.c3[q], r.c3[q + 1], p.vec_in_lo);
            ld_pair(hh + q, r.c4[q], r.c4[q + 1], p.vec_in_hi);
        }
        return;
    }
    int re, ro;
    bool rev, rov;
    if (MIRROR) {
        re = fold_ws(2 * vi, p.h) >> 1;
        ro = fold_ws(2 * vi + 1, p.h) >> 1;
        rev = rov = true;
    } else {
        rev = (vi >= 0) && (vi < p.hq);
        rov = (vi >= 0) && (vi < p.hh);
        re = rev ? vi : 0;
        ro = rov ? vi : 0;
    }
    // defensive clamps keep every address inside the bands (the checked build
    // reports a row that needed one)
    dev_in(p.status, !rev || (re >= 0 && re < p.hq));
    dev_in(p.status, !rov || (ro >= 0 && ro < p.hh));
    re = min(max(re, 0), p.hq - 1);
    ro = min(max(ro, 0), max(p.hh - 1, 0));
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int j = jb + q;
        int ce, co;
        bool cev, cov;
        if (MIRROR) {
            ce = fold_ws(2 * j, p.w) >> 1;
            co = fold_ws(2 * j + 1, p.w) >> 1;
            cev = cov = true;
        } else {
            cev = (j >= 0) && (j < p.wq);
            cov = (j >= 0) && (j < p.wh);
            ce = cev ? j : 0;
            co = cov ? j : 0;
        }
        dev_in(p.status, !cev || (ce >= 0 && ce < p.wq));
        dev_in(p.status, !cov || (co >= 0 && co < p.wh));
        ce = min(max(ce, 0), p.wq - 1);
        co = min(max(co, 0), max(p.wh - 1, 0));
        CT v1, v2, v3, v4;
        if (p.ll_is_ct)
            v1 = reinterpret_cast<const CT*>(p.ll)[int64_t(re) * p.ll_pitch + ce];
        else
            v1 = ld_one<BT, CT>(reinterpret_cast<const BT*>(p.ll) + int64_t(re) * p.ll_pitch + ce);
        v2 = ld_one<BT, CT>(coef + int64_t(re) * p.coef_pitch + p.wq + co);
        v3 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + ce);
        v4 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + co);
        r.c1[q] = (rev && cev) ? v1 : CT(0);
        r.c2[q] = (rev && cov) ? v2 : CT(0);
        r.c3[q] = (rov && cev) ? v3 : CT(0);
        r.c4[q] = (rov && cov) ? v4 : CT(0);
    }
}

// L1 adjoint: the gradient of l1_scale * sum |detail| w.r.t. the coefficients
template <class CT, int QL>
__device__ __forceinline__ void l1_transform(const InvParams& p, Row<CT, QL>& r) {
    const float s = p.l1_scale_dev ? p.l1_scale * *p.l1_scale_dev : p.l1_scale;
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        if (!p.ll_is_ct) r.c1[q] = CT(0);  // the coarsest LL is not in the loss
        r.c2[q] = CT(r.c2[q] > 0 ? s : (r.c2[q] < 0 ? -s : 0.f));
        r.c3[q] = CT(r.c3[q] > 0 ? s : (r.c3[q] < 0 ? -s : 0.f));
        r.c4[q] = CT(r.c4[q] > 0 ? s : (r.c4[q] < 0 ? -s : 0.f));
    }
}

// --------------------------------------------------------- inverse / adjoint
// One unit (strip s, quad rows [R0, R1)) of one inverse level with direct
// band loads (any alignment).  Pipe: Inv97<S, QL>, Inv53<S, QL>, Inv137<S, QL>.
// BT: coefficient element type.
template <class Pipe, class BT, bool ADJ, int QL>
__device__ __forceinline__ void inv_unit(const InvParams& p, int s, int R0, int R1, int lane) {
    static_assert(!ADJ, "the adjoint runs the staged units with the extended domain");
    using CT = typename Pipe::CT;
    using R = Row<CT, QL>;
    constexpr bool MIRROR = !ADJ;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int OUTQ = 32 * QL - 2 * HQ;
    const int A0 = R0 - WARM;
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int x0 = s * (2 * OUTQ) - 2 * HQ;
    const int jb = x0 / 2 + QL * lane;
    // the whole strip reads only existing band columns
    const bool fast_cols = (x0 >= 0) && (x0 / 2 + 32 * QL <= p.wh);
    bool mine[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        mine[q] = (lq >= HQ) && (lq < 32 * QL - HQ);
    }

    Pipe pipe;
    pipe.init();
    auto fast_row = [&](int vi) { return fast_cols && vi >= 0 && 2 * vi + 1 < p.h; };

    R pf[2];  // rows vi+1 and vi+2 in flight
    load_bands<CT, BT, MIRROR, QL>(p, A0, jb, fast_row(A0), pf[0]);
    load_bands<CT, BT, MIRROR, QL>(p, A0 + 1, jb, fast_row(A0 + 1), pf[1]);
    if constexpr (ADJ) {
        if (p.l1) {
            l1_transform(p, pf[0]);
            l1_transform(p, pf[1]);
        }
    }
    CT* row_e = reinterpret_cast<CT*>(p.out) + int64_t(2 * R0) * p.out_pitch;
    const int px = 2 * jb;  // first pixel column of the lane
    for (int gi = 0; gi < n_grp; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            if (gi * PHASES + PH >= n_arr) return;
            const int vi = A0 + gi * PHASES + PH;
            pipe.template slot<PH>() = pf[PH % 2];
            load_bands<CT, BT, MIRROR, QL>(p, vi + 2, jb, fast_row(vi + 2), pf[PH % 2]);
            if constexpr (ADJ) {
                if (p.l1) l1_transform(p, pf[PH % 2]);
            }
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if (oi < R0 || oi >= R1) return;
            CT* row_o = row_e + p.out_pitch;
            const bool has_o = 2 * oi + 1 < p.h;
            const CT* out0 = reinterpret_cast<const CT*>(p.out);
#pragma unroll
            for (int q = 0; q < QL; q += 2) {
                const int c = px + 2 * q;
                if (mine[q] && mine[q + 1] && p.vec_out && c + 3 < p.w) {
                    if (dev_in_rect(p.status, row_e + c, out0, p.out_pitch, p.h, p.w, 4))
                        st4<CT>(row_e + c, out.c1[q], out.c2[q], out.c1[q + 1], out.c2[q + 1]);
                    if (has_o && dev_in_rect(p.status, row_o + c, out0, p.out_pitch, p.h, p.w, 4))
                        st4<CT>(row_o + c, out.c3[q], out.c4[q], out.c3[q + 1], out.c4[q + 1]);
                } else {
                    const CT ev[4] = {out.c1[q], out.c2[q], out.c1[q + 1], out.c2[q + 1]};
                    const CT od[4] = {out.c3[q], out.c4[q], out.c3[q + 1], out.c4[q + 1]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (mine[q + (k >> 1)] && c + k < p.w) {
                            if (dev_in_rect(p.status, row_e + c + k, out0, p.out_pitch, p.h, p.w, 1))
                                row_e[c + k] = ev[k];
                            if (has_o && dev_in_rect(p.status, row_o + c + k, out0, p.out_pitch, p.h, p.w, 1))
                                row_o[c + k] = od[k];
                        }
                    }
                }
            }
            row_e += 2 * p.out_pitch;
        });
    }
}

// cp.async of `bytes` (4 or 8) from global to shared memory; src_bytes 0
// zero-fills the destination.
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src, bool valid) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
                 "r"(valid ? BYTES : 0)
                 : "memory");
}

// 8 bytes to shared memory, the first n (0, 4 or 8) from global, the rest zero
__device__ __forceinline__ void cp_async_n8(void* dst, const void* src, int n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}

template <class T, class CT>
__device__ __forceinline__ void ld_pair_smem(const unsigned char* p, CT& a, CT& b) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x, b = v.y;
    } else if constexpr (std::is_same<T, int>::value) {
        const int2 v = *reinterpret_cast<const int2*>(p);
        a = v.x, b = v.y;
    } else if constexpr (std::is_same<T, __half>::value) {
        const __half2 v = *reinterpret_cast<const __half2*>(p);
        a = __low2float(v), b = __high2float(v);
    } else {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
        a = __low2float(v), b = __high2float(v);
    }
}

// Shared-memory ring of the staged inverse / adjoint: per stage QR quad rows
// of the four bands, 256 bytes per band row (the lane's two quads as one pair).
template <int QR, int NST, int NW>
constexpr size_t inv_smem_bytes() {
    return size_t(NW) * NST * QR * 4 * 256 + size_t(NW) * NST * 8;
}

// Where an adjoint output pixel (r, c) goes: the image, the side buffer (the
// four extended columns or rows past an edge), or nowhere (beyond them).
__device__ __forceinline__ void adj_route_store(const InvParams& p, float* img_row, int r, int c, float v) {
    if (c < -4 || c >= p.w + 4 || r < -4 || r >= p.h + 4) return;
    const bool rin = (r >= 0) && (r < p.h), cin = (c >= 0) && (c < p.w);
    const int64_t side_len = adj_side_floats(p.h, p.w);
    float* dst;
    if (rin && cin) {
        dst = img_row + c;
        if (!dev_in_rect(p.status, dst, static_cast<float*>(p.out), p.out_pitch, p.h, p.w, 1)) return;
    } else if (!cin) {  // extended column (corners too)
        dst = p.side + (r + 4) * 8 + (c < 0 ? c + 4 : 4 + c - p.w);
        if (!dev_in_span(p.status, dst, p.side, side_len, 1)) return;
    } else {  // extended row inside the columns
        dst = p.side + int64_t(8) * (p.h + 8) + int64_t(r < 0 ? r + 4 : 4 + r - p.h) * p.w + c;
        if (!dev_in_span(p.status, dst, p.side, side_len, 1)) return;
    }
    *dst = v;
}

// Stores of the adjoint units: plain (every output inside the image), routed
// by lane (ROUTE_EDGE: a lane's four output columns lie inside the image, in
// the four extended columns on one side, or beyond them, fixed for the unit;
// each pixel row of four goes as one vector store to the image, the side
// buffer's extended rows or its extended columns), or pixel by pixel
// (ROUTE_PIXELS, adj_route_store: lanes whose four columns straddle an edge).
enum { ROUTE_NONE = 0, ROUTE_EDGE = 1, ROUTE_PIXELS = 2 };
// column class of a lane's four output columns px .. px+3
enum { CC_IN = 0, CC_SIDE_L = 1, CC_SIDE_R = 2, CC_DROP = 3, CC_MIXED = 4 };

__device__ __forceinline__ int adj_col_class(const InvParams& p, int px) {
    if (px >= 0 && px + 3 < p.w) return CC_IN;
    if (px == -4) return CC_SIDE_L;
    if (px == p.w) return CC_SIDE_R;
    if (px + 3 < -4 || px >= p.w + 4) return CC_DROP;
    return CC_MIXED;
}

// one pixel row of four values of a lane of class cc (not CC_DROP); svec:
// the side buffer is 16-byte aligned
__device__ __forceinline__ void adj_edge_store(const InvParams& p, float* img_row, int r, int px, int cc, bool svec,
                                               const float (&v)[4]) {
    const bool rin = (r >= 0) && (r < p.h);
    const bool rext = !rin && (r >= -4) && (r < p.h + 4);
    if (!rin && !rext) return;
    float* dst;
    bool vec;
    if (cc == CC_IN) {
        if (rin) {
            dst = img_row + px;
            vec = p.vec_out;
        } else {
            dst = p.side + int64_t(8) * (p.h + 8) + int64_t(r < 0 ? r + 4 : 4 + r - p.h) * p.w + px;
            vec = svec && (p.w & 3) == 0;
        }
    } else if (cc != CC_MIXED) {  // the four extended columns of one side (corners too)
        dst = p.side + (r + 4) * 8 + (cc == CC_SIDE_L ? 0 : 4);
        vec = svec;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) adj_route_store(p, img_row, r, px + k, v[k]);
        return;
    }
    if constexpr (CHECKED_BUILD) {
        const bool ok = (cc == CC_IN && rin)
                            ? dev_in_rect(p.status, dst, static_cast<const float*>(p.out), p.out_pitch, p.h, p.w, 4)
                            : dev_in_span(p.status, dst, p.side, adj_side_floats(p.h, p.w), 4);
        if (!ok) return;
    }
    if (vec) {
        st4<float>(dst, v[0], v[1], v[2], v[3]);
    } else {
        dst[0] = v[0], dst[1] = v[1], dst[2] = v[2], dst[3] = v[3];
    }
}

// The two pixel rows of one quad row of a ROUTE_EDGE lane, out of line: the
// row loop keeps only its common case (both rows and every lane's columns
// inside the image) and branches here around it.
static __device__ __noinline__ void adj_edge_store_rows(const InvParams& p, float* row_e, int r, int px, int cc, bool svec,
                                                 float e0, float e1, float e2, float e3, float o0, float o1, float o2,
                                                 float o3) {
    if (cc == CC_DROP) return;
    const float ev[4] = {e0, e1, e2, e3}, od[4] = {o0, o1, o2, o3};
    adj_edge_store(p, row_e, r, px, cc, svec, ev);
    adj_edge_store(p, row_e + p.out_pitch, r + 1, px, cc, svec, od);
}

// one pixel row of four values of a ROUTE_PIXELS lane whose columns all lie
// inside the image
__device__ __forceinline__ void adj_row_store(const InvParams& p, float* img_row, int r, int px, const float (&v)[4]) {
    adj_edge_store(p, img_row, r, px, CC_IN, (reinterpret_cast<uintptr_t>(p.side) & 15) == 0, v);
}

// One unit of a strip: the bands stream through a ring of NST stages of QR
// quad rows filled by cp.async (mirrored rows for the inverse, zero rows for
// the adjoint at the top and bottom).  Interior strips copy each lane's quad
// pair at once; EDGE strips (the first and last of a row, 4-byte types) copy
// element by element from the mirrored (inverse) or zero-filled (adjoint)
// columns.  The adjoint's units lie on the extended domain (p.ext quads and
// quad rows past every edge; strip s starts 2 * p.ext pixels further left);
// its ROUTE_EDGE units copy quad pairs too, zero-filled where a pair lies
// past a band's last column (a pair of an odd-width band that straddles it
// copies its first element alone), and route their stores.  Returns false
// when a stage wait timed out.
template <class Pipe, class BT, bool ADJ, int QR, int NST, bool EDGE, int ROUTE = ROUTE_NONE>
__device__ __forceinline__ bool inv_unit_staged(const InvParams& p, int s, int R0, int R1, int lane,
                                                unsigned char* ring, uint64_t* bars, uint32_t& gstage) {
    using CT = typename Pipe::CT;
    using R = Row<CT, 2>;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int QL = 2, OUTQ = 32 * QL - 2 * HQ;
    constexpr int BAND = 256, ROWB = 4 * BAND, STAGEB = QR * ROWB;
    constexpr int PB = 2 * int(sizeof(BT));  // bytes of a coefficient pair
    static_assert(PHASES % QR == 0, "a group of arrivals must cover whole stages");
    static_assert(HQ % 2 == 0, "a lane's two quads are both output or both halo");
    static_assert(ROUTE == ROUTE_NONE || ADJ, "routed stores belong to the adjoint");
    static_assert(ROUTE != ROUTE_EDGE || (!EDGE && PB == 8), "routed edge units copy FP32 pairs");
    const int A0 = R0 - WARM;
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int NT = (n_arr + QR - 1) / QR;
    const int x0 = s * (2 * OUTQ) - 2 * HQ - (ADJ ? 2 * p.ext : 0);
    const int jb = x0 / 2 + QL * lane;
    const bool mine = (lane >= HQ / 2) && (lane < 32 - HQ / 2);
    const BT* coef = reinterpret_cast<const BT*>(p.coef);

    // EDGE: every lane copies its band elements one by one (4-byte types), at
    // the mirrored (inverse) or zero-filled (adjoint) columns
    int ce[2], co[2];
    bool cev[2], cov[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = jb + q;
        if (ADJ) {
            cev[q] = (j >= 0) && (j < p.wq);
            cov[q] = (j >= 0) && (j < p.wh);
            ce[q] = cev[q] ? j : 0;
            co[q] = cov[q] ? j : 0;
        } else {
            ce[q] = fold_ws(2 * j, p.w) >> 1;
            co[q] = fold_ws(2 * j + 1, p.w) >> 1;
            cev[q] = cov[q] = true;
        }
        ce[q] = min(max(ce[q], 0), p.wq - 1);
        co[q] = min(max(co[q], 0), max(p.wh - 1, 0));
    }
    // ROUTE_EDGE: bytes of the lane's pair copied from the even-column (LL,
    // LH) and odd-column (HL, HH) bands: 8 (both inside), 4 (the first only:
    // the last column of an odd-width band) or 0, the rest zero-filled
    int nbe = 8, nbo = 8, je = jb, jo = jb, cc = CC_IN;
    bool svec = false;
    if constexpr (ROUTE == ROUTE_EDGE) {
        nbe = jb < 0 ? 0 : (jb + 1 < p.wq ? 8 : (jb < p.wq ? 4 : 0));
        nbo = jb < 0 ? 0 : (jb + 1 < p.wh ? 8 : (jb < p.wh ? 4 : 0));
        je = nbe ? jb : 0;
        jo = nbo ? jb : 0;
        cc = mine ? adj_col_class(p, 2 * jb) : CC_DROP;
        svec = (reinterpret_cast<uintptr_t>(p.side) & 15) == 0;
    }
    // every output lane's four columns inside the image (warp-uniform)
    const bool cols_in = ROUTE == ROUTE_EDGE && __all_sync(0xffffffffu, cc == CC_IN || cc == CC_DROP);
    // checked build: the bands as rectangles (LL hq x wq, HL hq x wh, LH hh x
    // wq, HH hh x wh) and the output image (h x w) that every access must fall in
    const CT* ll0c = reinterpret_cast<const CT*>(p.ll);
    const BT* ll0b = reinterpret_cast<const BT*>(p.ll);
    const BT* hl0 = coef + p.wq;
    const BT* lh0 = coef + int64_t(p.hq) * p.coef_pitch;
    const BT* hh0 = lh0 + p.wq;
    const CT* out0 = reinterpret_cast<const CT*>(p.out);
    (void)ll0c, (void)ll0b, (void)hl0, (void)lh0, (void)hh0, (void)out0;
    auto issue = [&](int t, int slot) {
        unsigned char* st = ring + slot * STAGEB;
#pragma unroll
        for (int r = 0; r < QR; ++r) {
            const int vi = A0 + t * QR + r;
            int re, ro;
            bool rev, rov;
            if (ADJ) {
                rev = (vi >= 0) && (vi < p.hq);
                rov = (vi >= 0) && (vi < p.hh);
                re = rev ? vi : 0;
                ro = rov ? vi : 0;
            } else {
                const bool in = (vi >= 0) && (2 * vi + 1 < p.h);
                re = in ? vi : (fold_ws(2 * vi, p.h) >> 1);
                ro = in ? vi : (fold_ws(2 * vi + 1, p.h) >> 1);
                rev = rov = true;
            }
            unsigned char* d = st + r * ROWB;
            if constexpr (EDGE) {
                static_assert(sizeof(BT) == 4 && sizeof(CT) == 4, "element copies of 4-byte types");
                const CT* llr = reinterpret_cast<const CT*>(p.ll) + int64_t(re) * p.ll_pitch;
                const BT* hlr = coef + int64_t(re) * p.coef_pitch + p.wq;
                const BT* lhr = coef + int64_t(p.hq + ro) * p.coef_pitch;
                const BT* hhr = lhr + p.wq;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    bool v_ll = rev && cev[q], v_hl = rev && cov[q], v_lh = rov && cev[q], v_hh = rov && cov[q];
                    if constexpr (CHECKED_BUILD) {
                        v_ll = v_ll && dev_in_rect(p.status, llr + ce[q], ll0c, p.ll_pitch, p.hq, p.wq, 1);
                        v_hl = v_hl && dev_in_rect(p.status, hlr + co[q], hl0, p.coef_pitch, p.hq, p.wh, 1);
                        v_lh = v_lh && dev_in_rect(p.status, lhr + ce[q], lh0, p.coef_pitch, p.hh, p.wq, 1);
                        v_hh = v_hh && dev_in_rect(p.status, hhr + co[q], hh0, p.coef_pitch, p.hh, p.wh, 1);
                    }
                    cp_async_small<4>(d + lane * 8 + q * 4, llr + ce[q], v_ll);
                    cp_async_small<4>(d + BAND + lane * 8 + q * 4, hlr + co[q], v_hl);
                    cp_async_small<4>(d + 2 * BAND + lane * 8 + q * 4, lhr + ce[q], v_lh);
                    cp_async_small<4>(d + 3 * BAND + lane * 8 + q * 4, hhr + co[q], v_hh);
                }
            } else if constexpr (ROUTE == ROUTE_EDGE) {
                const void* llr = p.ll_is_ct ? static_cast<const void*>(reinterpret_cast<const CT*>(p.ll) +
                                                                         int64_t(re) * p.ll_pitch + je)
                                             : static_cast<const void*>(reinterpret_cast<const BT*>(p.ll) +
                                                                         int64_t(re) * p.ll_pitch + je);
                const BT* hlr = coef + int64_t(re) * p.coef_pitch + p.wq + jo;
                const BT* lhr = coef + int64_t(p.hq + ro) * p.coef_pitch + je;
                const BT* hhr = coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + jo;
                int n_ll = rev ? nbe : 0, n_hl = rev ? nbo : 0, n_lh = rov ? nbe : 0, n_hh = rov ? nbo : 0;
                if constexpr (CHECKED_BUILD) {
                    const bool ll_ok = p.ll_is_ct ? dev_in_rect(p.status, static_cast<const CT*>(llr), ll0c, p.ll_pitch,
                                                                p.hq, p.wq, n_ll / 4)
                                                  : dev_in_rect(p.status, static_cast<const BT*>(llr), ll0b, p.ll_pitch,
                                                                p.hq, p.wq, n_ll / 4);
                    n_ll = (n_ll == 0 || ll_ok) ? n_ll : 0;
                    n_hl = (n_hl == 0 || dev_in_rect(p.status, hlr, hl0, p.coef_pitch, p.hq, p.wh, n_hl / 4)) ? n_hl : 0;
                    n_lh = (n_lh == 0 || dev_in_rect(p.status, lhr, lh0, p.coef_pitch, p.hh, p.wq, n_lh / 4)) ? n_lh : 0;
                    n_hh = (n_hh == 0 || dev_in_rect(p.status, hhr, hh0, p.coef_pitch, p.hh, p.wh, n_hh / 4)) ? n_hh : 0;
                }
                cp_async_n8(d + lane * 8, llr, n_ll);
                cp_async_n8(d + BAND + lane * 8, hlr, n_hl);
                cp_async_n8(d + 2 * BAND + lane * 8, lhr, n_lh);
                cp_async_n8(d + 3 * BAND + lane * 8, hhr, n_hh);
            } else {
                const CT* llc = reinterpret_cast<const CT*>(p.ll) + int64_t(re) * p.ll_pitch + jb;
                const BT* llb = reinterpret_cast<const BT*>(p.ll) + int64_t(re) * p.ll_pitch + jb;
                const BT* hlr = coef + int64_t(re) * p.coef_pitch + p.wq + jb;
                const BT* lhr = coef + int64_t(p.hq + ro) * p.coef_pitch + jb;
                const BT* hhr = coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + jb;
                bool v_ll = rev, v_hl = rev, v_lh = rov, v_hh = rov;
                if constexpr (CHECKED_BUILD) {
                    v_ll = v_ll && (p.ll_is_ct ? dev_in_rect(p.status, llc, ll0c, p.ll_pitch, p.hq, p.wq, 2)
                                               : dev_in_rect(p.status, llb, ll0b, p.ll_pitch, p.hq, p.wq, 2));
                    v_hl = v_hl && dev_in_rect(p.status, hlr, hl0, p.coef_pitch, p.hq, p.wh, 2);
                    v_lh = v_lh && dev_in_rect(p.status, lhr, lh0, p.coef_pitch, p.hh, p.wq, 2);
                    v_hh = v_hh && dev_in_rect(p.status, hhr, hh0, p.coef_pitch, p.hh, p.wh, 2);
                }
                if (p.ll_is_ct)
                    cp_async_small<8>(d + lane * 8, llc, v_ll);
                else
                    cp_async_small<PB>(d + lane * PB, llb, v_ll);
                cp_async_small<PB>(d + BAND + lane * PB, hlr, v_hl);
                cp_async_small<PB>(d + 2 * BAND + lane * PB, lhr, v_lh);
                cp_async_small<PB>(d + 3 * BAND + lane * PB, hhr, v_hh);
            }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&bars[slot]))
                     : "memory");
    };
    for (int t = 0; t < NST && t < NT; ++t) issue(t, (gstage + t) % NST);

    Pipe pipe;
    pipe.init();
    bool ok = true;
    int t = 0, slot = 0;
    const unsigned char* stage = ring;
    CT* row_e = reinterpret_cast<CT*>(p.out) + int64_t(2 * R0) * p.out_pitch;
    const int px = 2 * jb;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            constexpr int QI = PH % QR;
            if (gi * PHASES + PH >= QR * NT) return;
            if constexpr (QI == 0) {
                if (!ok) return;
                const uint32_t gs = gstage + t;
                slot = gs % NST;
                if (!mbar_wait_bounded(&bars[slot], (gs / NST) & 1u, p.status, p.timeout_ns)) {
                    for (int u = t + 1; u < NT && u < t + NST; ++u) {
                        const uint32_t gu = gstage + u;
                        mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, p.timeout_ns);
                    }
                    ok = false;
                    return;
                }
                stage = ring + slot * STAGEB;
            }
            const int vi = A0 + gi * PHASES + PH;
            R& in = pipe.template slot<PH>();
            const unsigned char* d = stage + QI * ROWB;
            if (p.ll_is_ct)
                ld_pair_smem<CT, CT>(d + lane * 8, in.c1[0], in.c1[1]);
            else
                ld_pair_smem<BT, CT>(d + lane * PB, in.c1[0], in.c1[1]);
            ld_pair_smem<BT, CT>(d + BAND + lane * PB, in.c2[0], in.c2[1]);
            ld_pair_smem<BT, CT>(d + 2 * BAND + lane * PB, in.c3[0], in.c3[1]);
            ld_pair_smem<BT, CT>(d + 3 * BAND + lane * PB, in.c4[0], in.c4[1]);
            if constexpr (ADJ) {
                if (p.l1) l1_transform(p, in);
            }
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if constexpr (ROUTE == ROUTE_EDGE) {
                if (oi >= R0 && oi < R1) {
                    if (cols_in && oi >= 0 && 2 * oi + 1 < p.h) {  // warp-uniform
                        if (cc == CC_IN && (!CHECKED_BUILD ||
                                            (dev_in_rect(p.status, row_e + px, out0, p.out_pitch, p.h, p.w, 4) &&
                                             dev_in_rect(p.status, row_e + p.out_pitch + px, out0, p.out_pitch, p.h,
                                                         p.w, 4)))) {
                            CT* row_o = row_e + p.out_pitch;
                            if (p.vec_out) {
                                st4<CT>(row_e + px, out.c1[0], out.c2[0], out.c1[1], out.c2[1]);
                                st4<CT>(row_o + px, out.c3[0], out.c4[0], out.c3[1], out.c4[1]);
                            } else {
                                row_e[px] = out.c1[0], row_e[px + 1] = out.c2[0];
                                row_e[px + 2] = out.c1[1], row_e[px + 3] = out.c2[1];
                                row_o[px] = out.c3[0], row_o[px + 1] = out.c4[0];
                                row_o[px + 2] = out.c3[1], row_o[px + 3] = out.c4[1];
                            }
                        }
                    } else {
                        adj_edge_store_rows(p, row_e, 2 * oi, px, cc, svec, out.c1[0], out.c2[0], out.c1[1],
                                            out.c2[1], out.c3[0], out.c4[0], out.c3[1], out.c4[1]);
                    }
                    row_e += 2 * p.out_pitch;
                }
            } else if constexpr (ROUTE == ROUTE_PIXELS) {
                if (oi >= R0 && oi < R1 && mine) {
                    const CT ev[4] = {out.c1[0], out.c2[0], out.c1[1], out.c2[1]};
                    const CT od[4] = {out.c3[0], out.c4[0], out.c3[1], out.c4[1]};
                    CT* row_o = row_e + p.out_pitch;
                    if (px >= 0 && px + 3 < p.w) {  // the lane's columns inside: whole pixel rows
                        adj_row_store(p, row_e, 2 * oi, px, ev);
                        adj_row_store(p, row_o, 2 * oi + 1, px, od);
                    } else {
#pragma unroll
                        for (int k2 = 0; k2 < 4; ++k2) {
                            adj_route_store(p, row_e, 2 * oi, px + k2, ev[k2]);
                            adj_route_store(p, row_o, 2 * oi + 1, px + k2, od[k2]);
                        }
                    }
                }
                if (oi >= R0 && oi < R1) row_e += 2 * p.out_pitch;
            } else if (oi >= R0 && oi < R1) {
                CT* row_o = row_e + p.out_pitch;
                const bool has_o = 2 * oi + 1 < p.h;
                if (mine && p.vec_out && px + 3 < p.w) {
                    if (dev_in_rect(p.status, row_e + px, out0, p.out_pitch, p.h, p.w, 4))
                        st4<CT>(row_e + px, out.c1[0], out.c2[0], out.c1[1], out.c2[1]);
                    if (has_o && dev_in_rect(p.status, row_o + px, out0, p.out_pitch, p.h, p.w, 4))
                        st4<CT>(row_o + px, out.c3[0], out.c4[0], out.c3[1], out.c4[1]);
                } else if (mine) {
                    const CT ev[4] = {out.c1[0], out.c2[0], out.c1[1], out.c2[1]};
                    const CT od[4] = {out.c3[0], out.c4[0], out.c3[1], out.c4[1]};
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        if (px + k2 < p.w) {
                            if (dev_in_rect(p.status, row_e + px + k2, out0, p.out_pitch, p.h, p.w, 1))
                                row_e[px + k2] = ev[k2];
                            if (has_o && dev_in_rect(p.status, row_o + px + k2, out0, p.out_pitch, p.h, p.w, 1))
                                row_o[px + k2] = od[k2];
                        }
                    }
                }
                row_e += 2 * p.out_pitch;
            }
            if constexpr (QI == QR - 1) {
                __syncwarp();
                if (ok && t + NST < NT) issue(t + NST, slot);
                ++t;
            }
        });
    }
    if (ok) gstage += NT;
    return ok;
}

// UNITS_INNER: staged pair copies, plain stores.  UNITS_EDGE of the inverse:
// staged element copies from mirrored columns (4-byte types) or direct loads;
// of the adjoint (one pipeline, Adj97, on the extended domain): pair copies
// with zero fill and stores routed by lane when the bands are pair-aligned,
// else element copies and stores routed by pixel.
template <class Pipe, class BT, bool ADJ, int QR, int NST, int CLS>
__device__ __forceinline__ bool inv_unit_any(const InvParams& p, int s, int R0, int R1, int lane,
                                             unsigned char* ring, uint64_t* bars, uint32_t& gstage) {
    static_assert(CLS == UNITS_INNER || CLS == UNITS_EDGE, "a level runs its inner and edge units in two launches");
    const bool staged = p.vec_in_lo && p.vec_in_hi && p.vec_ll;
    if constexpr (CLS == UNITS_INNER) {
        return inv_unit_staged<Pipe, BT, ADJ, QR, NST, false>(p, s, R0, R1, lane, ring, bars, gstage);
    } else if constexpr (ADJ) {
        if (staged)
            return inv_unit_staged<Pipe, BT, true, QR, NST, false, ROUTE_EDGE>(p, s, R0, R1, lane, ring, bars, gstage);
        return inv_unit_staged<Pipe, BT, true, QR, NST, true, ROUTE_PIXELS>(p, s, R0, R1, lane, ring, bars, gstage);
    } else {
        if constexpr (sizeof(BT) == 4) {
            if (staged) return inv_unit_staged<Pipe, BT, false, QR, NST, true>(p, s, R0, R1, lane, ring, bars, gstage);
        }
        inv_unit<Pipe, BT, false, 2>(p, s, R0, R1, lane);
        return true;
    }
}

template <int QR, int NST, int NW>
__device__ __forceinline__ void inv_ring(unsigned char* smem, int warp, int lane, unsigned char*& ring,
                                         uint64_t*& bars) {
    ring = smem + size_t(warp) * NST * QR * 4 * 256;
    bars = reinterpret_cast<uint64_t*>(smem + size_t(NW) * NST * QR * 4 * 256) + warp * NST;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 32);
        fence_mbar_init();
    }
    __syncwarp();
}

// resident blocks the kernels of the two-quad-halo pipelines (CDF 9/7,
// CDF 5/3) are held to: the inner row loop fits the register budget of five
// 4-warp blocks per SM, the edge loops (element copies, predicated copies and
// routed stores) that of four; the DD 13/7 pipelines (six-row rings) are left
// to the compiler
template <class Pipe, int CLS>
struct InvMinBlocks {
    static constexpr int value = PipeGeom<Pipe>::HALO == 2 ? (CLS == UNITS_INNER ? 5 : 4) : 1;
};

// Strip s and quad rows [R0, R1) of the class's unit lu (on the extended
// domain of the adjoint); false for an empty piece of an edge unit.
__device__ __forceinline__ bool inv_unit_rows(const InvParams& p, int cls, int lu, int& s, int& R0, int& R1) {
    int g, k;
    inv_class_unit(p, cls, lu, s, g, k);
    R0 = g * p.seg_rows - p.ext;
    R1 = min(R0 + p.seg_rows, p.hq + p.ext);
    if (cls == UNITS_EDGE && inv_edge_split(p) > 1) {
        const int pr = (p.seg_rows + inv_edge_split(p) - 1) / inv_edge_split(p);
        R0 += k * pr;
        R1 = min(R1, R0 + pr);
    }
    return R0 < R1;
}

// Launch order.  The first launch of a level (the inner units of its first
// group of images for the inverse, the edge units for the adjoint) is a
// plain launch: stream order completes everything before it.  The level's
// later launches (the other unit class, later groups) share no data with the
// launches before them and are programmatic dependents that start as soon as
// those have placed all their blocks; none of them waits on the device.
// One level of one image: the units of class CLS, dealt round-robin.
template <class Pipe, class BT, bool ADJ, int QL, int NW, int CLS>
__global__ void __launch_bounds__(NW * 32, InvMinBlocks<Pipe, CLS>::value) inv_kernel(const InvParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ring;
    uint64_t* bars;
    inv_ring<INV_QR, INV_NST, NW>(smem, warp, lane, ring, bars);
    griddep_launch_dependents();
    uint32_t gstage = 0;
    const int n = inv_class_units(p, CLS);
    for (int lu = blockIdx.x * NW + warp; lu < n; lu += gridDim.x * NW) {
        int s, R0, R1;
        if (!inv_unit_rows(p, CLS, lu, s, R0, R1)) continue;
        if (!inv_unit_any<Pipe, BT, ADJ, INV_QR, INV_NST, CLS>(p, s, R0, R1, lane, ring, bars, gstage) ||
            dev_check_tripped(p.status))
            return;
    }
}

// One level of a group of images (InvGroupLaunch): the units of class CLS of
// every image, in order, the image found by binary search over the group's
// unit ranges.
template <class Pipe, class BT, bool ADJ, int QL, int NW, int CLS>
__global__ void __launch_bounds__(NW * 32, InvMinBlocks<Pipe, CLS>::value)
    inv_group_kernel(const __grid_constant__ InvGroupLaunch L) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ring;
    uint64_t* bars;
    inv_ring<INV_QR, INV_NST, NW>(smem, warp, lane, ring, bars);
    griddep_launch_dependents();
    uint32_t gstage = 0;
    for (int u = blockIdx.x * NW + warp; u < L.n_units[CLS]; u += gridDim.x * NW) {
        int lo = 0, hi = L.n_img - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.img[mid].u_begin[CLS] <= u) lo = mid;
            else hi = mid - 1;
        }
        const InvParams& p = L.img[lo].p;
        int s, R0, R1;
        if (!inv_unit_rows(p, CLS, u - L.img[lo].u_begin[CLS], s, R0, R1)) continue;
        if (!inv_unit_any<Pipe, BT, ADJ, INV_QR, INV_NST, CLS>(p, s, R0, R1, lane, ring, bars, gstage) ||
            dev_check_tripped(p.status))
            return;
    }
}

// ---------------------------------------------------------------- adjoint fold
// E^T of one adjoint level: every image pixel within five of an edge (the
// whole image when a side is at most ten) adds the side-buffer values of the
// extended positions whose whole-sample mirror it is: extended columns of its
// row, extended rows of its column, and both at once (corners).  One thread
// per such pixel, so no two threads write the same pixel.
// slot (0..7) of the extended position whose mirror is c in a side of n > 10
// samples, or -1: the mirror of -k is k, that of n-1+k is n-1-k (k = 1..4)
__device__ __forceinline__ int adj_mirror_slot(int c, int n) {
    if (c >= 1 && c <= 4) return 4 - c;
    if (c >= n - 5 && c <= n - 2) return n + 2 - c;
    return -1;
}

__device__ __forceinline__ void adj_fold_pixel(const InvParams& p, int r, int c) {
    const float* L = p.side;
    const float* T = p.side + int64_t(8) * (p.h + 8);
    float* o = reinterpret_cast<float*>(p.out) + int64_t(r) * p.out_pitch + c;
    if (!dev_in_rect(p.status, o, static_cast<const float*>(p.out), p.out_pitch, p.h, p.w, 1)) return;
    if constexpr (CHECKED_BUILD) {  // every side slot read below lies in the side buffer
        if (!dev_in(p.status, r >= 0 && r < p.h && c >= 0 && c < p.w)) return;
    }
    if (p.h > 10 && p.w > 10) {  // at most one source of each kind
        const int kc = adj_mirror_slot(c, p.w), kr = adj_mirror_slot(r, p.h);
        float acc = 0.f;
        if (kc >= 0) acc += L[(r + 4) * 8 + kc];
        if (kr >= 0) acc += T[int64_t(kr) * p.w + c];
        if (kc >= 0 && kr >= 0) acc += L[(kr < 4 ? kr : p.h + kr) * 8 + kc];
        if (kc >= 0 || kr >= 0) *o += acc;
        return;
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int pc = k < 4 ? k - 4 : p.w + (k - 4);  // extended column
        const int pr = k < 4 ? k - 4 : p.h + (k - 4);  // extended row
        const bool col_here = fold_ws(pc, p.w) == c;
        const bool row_here = fold_ws(pr, p.h) == r;
        if (col_here) acc += L[(r + 4) * 8 + k];  // extended column of this row
        if (row_here) acc += T[int64_t(k) * p.w + c];  // extended row of this column
        if (row_here) {
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) {  // corners: extended row and column
                const int pc2 = kc < 4 ? kc - 4 : p.w + (kc - 4);
                if (fold_ws(pc2, p.w) == c) acc += L[(pr + 4) * 8 + kc];
            }
        }
    }
    *o += acc;
}

// the pixels within five of an edge, as one index range: the first and last
// min(5, h) rows whole, then the first and last min(5, w) columns of the rows
// between
__host__ __device__ inline int adj_fold_count(int h, int w) {
    const int br = h <= 10 ? h : 10, bc = w <= 10 ? w : 10;
    return br * w + (h - br) * bc;
}
__device__ __forceinline__ void adj_fold_index(int h, int w, int i, int& r, int& c) {
    const int br = h <= 10 ? h : 10, bc = w <= 10 ? w : 10;
    if (i < br * w) {
        const int rr = i / w;
        r = rr < 5 || h <= 10 ? rr : h - 10 + rr;
        c = i % w;
        return;
    }
    i -= br * w;
    r = 5 + i / bc;
    const int cc = i % bc;
    c = cc < 5 || w <= 10 ? cc : w - 10 + cc;
}

}  // namespace dwt2
